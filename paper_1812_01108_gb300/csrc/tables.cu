// Residue tables of the full-atom model (paper Section 2): rigid groups and the
// standard-frame positions r0 of their atoms, built once on the host.
//
// The paper prints the transform structure (M_1 = M_0 R_1(phi), side chain
// through R' and R(chi), M_3 = M_1 R_3(psi), M_4 = M_3 R_4(omega)), the angle
// of R' (122.686 degrees) and the backbone constants, but no side-chain
// geometry.  The internal coordinates below are authored from ideal
// stereochemistry (bond lengths and angles of Engh & Huber, Acta Cryst. A47 (1991)
// 392-400); the HIS ring angles at ND1 and CD2 and the proline ring's fixed
// chi1 and CD dihedral are fitted so that those rings close at the Engh &
// Huber closure values.  Each side-chain atom is (group, bonded atom p, angle atom q,
// dihedral atom r, bond, angle, dihedral); indices count N=0, CA=1, C=2, O=3,
// then the side chain in output order.  A dihedral marked on_chi is an offset
// added to its group's chi.  The first atom of each group is the group's
// origin; group k's frame is S_k = S_{k-1} R(chi_k, pi - angle, bond) with
// S_0 = M_1 R'.
#include <math.h>
#include <string.h>

#include <mutex>

#include "tables.h"

namespace tpl {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;

struct IC {
    const char* name;
    int grp, p, q, r;
    double bond, ang, dih;
    int on_chi;
};

struct ResDef {
    const char* three;
    int n_chi, n_groups;
    double fixed_chi[kMaxGroups];
    int n_side;
    IC side[kMaxSide];
};

const ResDef kRes[kNumAminoAcids] = {
    {"ALA", 0, 1, {0.0}, 1, {{"CB", 1, 1, 0, 2, 1.521, 110.4, 0.0, 0}}},
    {"ARG", 4, 4, {0}, 7,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.520, 114.1, 0.0, 1},
      {"CD", 3, 5, 4, 1, 1.520, 111.3, 0.0, 1},
      {"NE", 4, 6, 5, 4, 1.460, 112.0, 0.0, 1},
      {"CZ", 4, 7, 6, 5, 1.329, 124.2, 0.0, 1},
      {"NH1", 4, 8, 7, 6, 1.326, 120.0, 0.0, 0},
      {"NH2", 4, 8, 7, 6, 1.326, 120.0, 180.0, 0}}},
    {"ASN", 2, 2, {0}, 4,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.516, 112.6, 0.0, 1},
      {"OD1", 2, 5, 4, 1, 1.231, 120.8, 0.0, 1},
      {"ND2", 2, 5, 4, 1, 1.328, 116.4, 180.0, 1}}},
    {"ASP", 2, 2, {0}, 4,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.516, 112.6, 0.0, 1},
      {"OD1", 2, 5, 4, 1, 1.249, 118.4, 0.0, 1},
      {"OD2", 2, 5, 4, 1, 1.249, 118.4, 180.0, 1}}},
    {"CYS", 1, 1, {0}, 2,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"SG", 1, 4, 1, 0, 1.808, 114.4, 0.0, 1}}},
    {"GLN", 3, 3, {0}, 5,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.520, 114.1, 0.0, 1},
      {"CD", 3, 5, 4, 1, 1.516, 112.6, 0.0, 1},
      {"OE1", 3, 6, 5, 4, 1.231, 120.8, 0.0, 1},
      {"NE2", 3, 6, 5, 4, 1.328, 116.4, 180.0, 1}}},
    {"GLU", 3, 3, {0}, 5,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.520, 114.1, 0.0, 1},
      {"CD", 3, 5, 4, 1, 1.516, 112.6, 0.0, 1},
      {"OE1", 3, 6, 5, 4, 1.249, 118.4, 0.0, 1},
      {"OE2", 3, 6, 5, 4, 1.249, 118.4, 180.0, 1}}},
    {"GLY", 0, 0, {0}, 0, {}},
    {"HIS", 2, 2, {0}, 6,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.497, 113.8, 0.0, 1},
      {"ND1", 2, 5, 4, 1, 1.378, 122.7, 0.0, 1},
      {"CD2", 2, 5, 4, 1, 1.354, 131.0, 180.0, 1},
      {"CE1", 2, 6, 5, 4, 1.345, 106.9, 180.0, 0},
      {"NE2", 2, 7, 5, 4, 1.382, 109.6, 180.0, 0}}},
    {"ILE", 2, 2, {0}, 4,
     {{"CB", 1, 1, 0, 2, 1.540, 111.5, 0.0, 0},
      {"CG1", 2, 4, 1, 0, 1.530, 110.4, 0.0, 1},
      {"CG2", 1, 4, 1, 0, 1.521, 110.5, -122.6, 1},
      {"CD1", 2, 5, 4, 1, 1.513, 113.8, 0.0, 1}}},
    {"LEU", 2, 2, {0}, 4,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.530, 116.3, 0.0, 1},
      {"CD1", 2, 5, 4, 1, 1.521, 110.7, 0.0, 1},
      {"CD2", 2, 5, 4, 1, 1.521, 110.7, 122.7, 1}}},
    {"LYS", 4, 4, {0}, 5,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.520, 114.1, 0.0, 1},
      {"CD", 3, 5, 4, 1, 1.520, 111.3, 0.0, 1},
      {"CE", 4, 6, 5, 4, 1.520, 111.3, 0.0, 1},
      {"NZ", 4, 7, 6, 5, 1.489, 111.9, 0.0, 1}}},
    {"MET", 3, 3, {0}, 4,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.520, 114.1, 0.0, 1},
      {"SD", 3, 5, 4, 1, 1.803, 112.7, 0.0, 1},
      {"CE", 3, 6, 5, 4, 1.791, 100.9, 0.0, 1}}},
    {"PHE", 2, 2, {0}, 7,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.502, 113.8, 0.0, 1},
      {"CD1", 2, 5, 4, 1, 1.384, 120.7, 0.0, 1},
      {"CD2", 2, 5, 4, 1, 1.384, 120.7, 180.0, 1},
      {"CE1", 2, 6, 5, 4, 1.382, 120.7, 180.0, 0},
      {"CE2", 2, 7, 5, 4, 1.382, 120.7, 180.0, 0},
      {"CZ", 2, 8, 6, 5, 1.382, 120.0, 0.0, 0}}},
    {"PRO", 0, 1, {-28.0}, 3,
     {{"CB", 1, 1, 0, 2, 1.530, 103.0, 0.0, 0},
      {"CG", 1, 4, 1, 0, 1.492, 104.5, 0.0, 1},
      {"CD", 1, 5, 4, 1, 1.503, 106.1, 33.0, 0}}},
    {"SER", 1, 1, {0}, 2,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"OG", 1, 4, 1, 0, 1.417, 111.1, 0.0, 1}}},
    {"THR", 1, 1, {0}, 3,
     {{"CB", 1, 1, 0, 2, 1.540, 111.5, 0.0, 0},
      {"OG1", 1, 4, 1, 0, 1.433, 109.6, 0.0, 1},
      {"CG2", 1, 4, 1, 0, 1.521, 110.5, -120.0, 1}}},
    {"TRP", 2, 2, {0}, 10,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.498, 113.6, 0.0, 1},
      {"CD1", 2, 5, 4, 1, 1.365, 126.9, 0.0, 1},
      {"CD2", 2, 5, 4, 1, 1.433, 126.6, 180.0, 1},
      {"NE1", 2, 6, 5, 4, 1.374, 110.2, 180.0, 0},
      {"CE2", 2, 7, 5, 4, 1.409, 107.2, 180.0, 0},
      {"CE3", 2, 7, 5, 4, 1.398, 133.9, 0.0, 0},
      {"CZ2", 2, 9, 7, 5, 1.394, 122.4, 180.0, 0},
      {"CZ3", 2, 10, 7, 5, 1.382, 118.6, 180.0, 0},
      {"CH2", 2, 11, 9, 7, 1.368, 117.5, 0.0, 0}}},
    {"TYR", 2, 2, {0}, 8,
     {{"CB", 1, 1, 0, 2, 1.530, 110.5, 0.0, 0},
      {"CG", 2, 4, 1, 0, 1.512, 113.9, 0.0, 1},
      {"CD1", 2, 5, 4, 1, 1.389, 120.8, 0.0, 1},
      {"CD2", 2, 5, 4, 1, 1.389, 120.8, 180.0, 1},
      {"CE1", 2, 6, 5, 4, 1.382, 121.2, 180.0, 0},
      {"CE2", 2, 7, 5, 4, 1.382, 121.2, 180.0, 0},
      {"CZ", 2, 8, 6, 5, 1.378, 119.6, 0.0, 0},
      {"OH", 2, 10, 8, 6, 1.376, 119.9, 180.0, 0}}},
    {"VAL", 1, 1, {0}, 3,
     {{"CB", 1, 1, 0, 2, 1.540, 111.5, 0.0, 0},
      {"CG1", 1, 4, 1, 0, 1.521, 110.5, 0.0, 1},
      {"CG2", 1, 4, 1, 0, 1.521, 110.5, -122.9, 1}}},
};

// Residue code 20 places the backbone's N, CA and C only: a chain of such
// residues is the Section 3 model, so one batch can hold both models.
const ResDef kResBackbone = {"BB", 0, 0, {0.0}, 0, {}};
const ResDef& res_def(int code) { return code < kNumAminoAcids ? kRes[code] : kResBackbone; }

const char* kBackboneNames[4] = {"N", "CA", "C", "O"};

// Backbone, Section 3: theta = pi - {2.1186, 1.9391, 2.0610}, d = {1.330, 1.460, 1.525}
// for the transforms placing N (omega), CA (phi), C (psi).
const double kBbAngle[3] = {2.1186, 1.9391, 2.0610};
const double kBbBond[3] = {1.330, 1.460, 1.525};
// Backbone O: bonded to C, angle CA-C-O 120.1 deg, dihedral N-CA-C-O = psi + 180.
const double kOBond = 1.231, kOAngle = 120.1, kODih = 180.0;
// R' about x by -122.686 deg in the R_x convention of Section 3 (L chirality).
const double kRprime = -122.686;

struct V3 {
    double x, y, z;
};
V3 v_sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 v_add(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 v_mul(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double v_dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 v_cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3 v_unit(V3 a) { return v_mul(1.0 / sqrt(v_dot(a, a)), a); }

// Natural-extension placement (Parsons et al., J. Comput. Chem. 26 (2005) 1063):
// atom d bonded to c with |cd| = bond, angle bcd = ang, dihedral abcd = dih.
V3 nerf(V3 a, V3 b, V3 c, double bond, double ang, double dih) {
    V3 bc = v_unit(v_sub(c, b));
    V3 n = v_unit(v_cross(v_sub(b, a), bc));
    V3 m = v_cross(n, bc);
    double dx = -bond * cos(ang), dy = bond * sin(ang) * cos(dih), dz = bond * sin(ang) * sin(dih);
    return v_add(c, v_add(v_mul(dx, bc), v_add(v_mul(dy, m), v_mul(dz, n))));
}

// Atom bonded to a frame's origin whose dihedral is the frame's own angle plus
// `off`: R_x(off) R_y(pi - ang) (bond, 0, 0).
V3 frame_child(double bond, double ang, double off) {
    double th = kPi - ang;
    return {bond * cos(th), bond * sin(th) * sin(off), -bond * sin(th) * cos(off)};
}

struct Built {
    FaTable f;
    FaTableD d;
};

Built* g_built = nullptr;
std::once_flag g_once;

void build() {
    Built* B = new Built;
    memset(B, 0, sizeof(Built));
    FaTable& F = B->f;
    FaTableD& D = B->d;
    for (int k = 0; k < 3; ++k) {
        double th = kPi - kBbAngle[k];
        D.bb.ct[k] = cos(th);
        D.bb.st[k] = sin(th);
        D.bb.d[k] = kBbBond[k];
        F.bb.ct[k] = (float)D.bb.ct[k];
        F.bb.st[k] = (float)D.bb.st[k];
        F.bb.d[k] = (float)D.bb.d[k];
    }
    D.rp_c = cos(kRprime * kDeg);
    D.rp_s = sin(kRprime * kDeg);
    F.rp_c = (float)D.rp_c;
    F.rp_s = (float)D.rp_s;
    V3 o = frame_child(kOBond, kOAngle * kDeg, kODih * kDeg);
    F.o_r0 = make_float4((float)o.x, (float)o.y, (float)o.z, 3.f);
    D.bb.o[0] = o.x; D.bb.o[1] = o.y; D.bb.o[2] = o.z;
    F.bb.o[0] = (float)o.x; F.bb.o[1] = (float)o.y; F.bb.o[2] = (float)o.z;

    for (int t = 0; t < kNumTypes; ++t) {
        const ResDef& R = res_def(t);
        const int n_atoms = t == kBackboneCode ? 3 : 4 + R.n_side;  // no O on a backbone-only residue
        D.n_atoms[t] = F.n_atoms[t] = (uint8_t)n_atoms;
        D.n_chi[t] = F.n_chi[t] = (uint8_t)R.n_chi;
        D.n_groups[t] = F.n_groups[t] = (uint8_t)R.n_groups;
        // group ids and r0 of the backbone atoms
        D.group[t][0] = 0;
        D.group[t][1] = 1;
        D.group[t][2] = 2;
        D.group[t][3] = 2;
        D.r0[t][3][0] = o.x;
        D.r0[t][3][1] = o.y;
        D.r0[t][3][2] = o.z;
        // origin atom of each group; index 1 (CA) acts as the origin of group 0
        int origin[kMaxGroups + 1] = {1, -1, -1, -1, -1};
        for (int i = 0; i < R.n_side; ++i)
            if (origin[R.side[i].grp] < 0) origin[R.side[i].grp] = 4 + i;
        for (int k = 1; k <= R.n_groups; ++k) {
            const IC& e = R.side[origin[k] - 4];
            double th = kPi - e.ang * kDeg;
            D.grp_ct[t][k - 1] = cos(th);
            D.grp_st[t][k - 1] = sin(th);
            D.grp_d[t][k - 1] = e.bond;
            D.fixchi[t][k - 1] = R.fixed_chi[k - 1] * kDeg;
            D.origin[t][k - 1] = (uint8_t)origin[k];
            F.grp[t][k - 1] = make_float4((float)cos(th), (float)sin(th), (float)e.bond, 0.f);
            F.fixchi[t][k - 1] = make_float2((float)cos(R.fixed_chi[k - 1] * kDeg),
                                             (float)sin(R.fixed_chi[k - 1] * kDeg));
        }
        // local positions in each group's frame
        V3 local[kMaxAtoms];
        for (int i = 0; i < R.n_side; ++i) {
            const IC& e = R.side[i];
            const int idx = 4 + i, k = e.grp;
            const int prev1 = origin[k - 1];
            const int prev2 = (k >= 2) ? origin[k - 2] : 0;
            if (idx == origin[k]) {
                local[idx] = {0.0, 0.0, 0.0};
            } else if (e.p == origin[k] && e.q == prev1 && e.r == prev2) {
                local[idx] = frame_child(e.bond, e.ang * kDeg, e.dih * kDeg);
            } else {
                V3 ref[3];
                const int ids[3] = {e.r, e.q, e.p};
                for (int m = 0; m < 3; ++m)
                    ref[m] = (ids[m] == prev1) ? V3{-D.grp_d[t][k - 1], 0.0, 0.0} : local[ids[m]];
                local[idx] = nerf(ref[0], ref[1], ref[2], e.bond, e.ang * kDeg, e.dih * kDeg);
            }
            D.group[t][idx] = (uint8_t)(2 + k);
            D.r0[t][idx][0] = local[idx].x;
            D.r0[t][idx][1] = local[idx].y;
            D.r0[t][idx][2] = local[idx].z;
        }
        for (int i = 0; i < n_atoms; ++i) F.atom_grp[t][i] = D.group[t][i];
        for (int k = 1; k <= R.n_groups; ++k) F.origin[t][k - 1] = (uint8_t)origin[k];
        // side atoms sorted by group for the FP32 kernels
        int pos = 0;
        for (int k = 1; k <= R.n_groups; ++k) {
            for (int i = 0; i < R.n_side; ++i) {
                if (R.side[i].grp != k) continue;
                const int idx = 4 + i;
                F.side[t][pos++] = make_float4((float)local[idx].x, (float)local[idx].y,
                                               (float)local[idx].z, (float)(idx + 16 * k));
            }
            F.grp_end[t][k - 1] = (uint8_t)pos;
        }
    }
    g_built = B;
}

const Built& built() {
    std::call_once(g_once, build);
    return *g_built;
}

}  // namespace

const FaTable& fa_table() { return built().f; }
const FaTableD& fa_table_d() { return built().d; }
BackboneConst backbone_const() { return built().f.bb; }
BackboneConstD backbone_const_d() { return built().d.bb; }

const char* residue_three(int code) {
    return (code >= 0 && code < kNumTypes) ? res_def(code).three : nullptr;
}

const char* residue_atom_name(int code, int idx) {
    if (code < 0 || code >= kNumTypes) return nullptr;
    if (idx < 0 || idx >= fa_table().n_atoms[code]) return nullptr;
    return idx < 4 ? kBackboneNames[idx] : res_def(code).side[idx - 4].name;
}

}  // namespace tpl
