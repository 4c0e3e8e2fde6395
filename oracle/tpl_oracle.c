/*
 * Plain FP64 CPU oracle (see tpl_oracle.h).  TEST INFRASTRUCTURE ONLY: the
 * product path never calls it.
 *
 * Everything here is sequential, unblocked and written in the paper's
 * notation so that it can be checked against the text by eye:
 *   Section 2  full-atom model: R(alpha, theta, d) = R_y(theta) T_x(d) R_x(alpha),
 *              cumulative transforms M_1 = M_0 R_1(phi), side chain
 *              M_0 R_1 R' R_2(chi) ..., M_3 = M_1 R_3(psi), M_4 = M_3 R_4(omega),
 *              atoms r = M r0, and the adjoint of Eq. 1.
 *   Section 3  backbone model: explicit R matrix, atom index rule and
 *              constants, M_i = R_0 ... R_i, derivative
 *              M_{3j} dR_{3j+1} M_{3j+1}^{-1} M_i 0, sums of Eq. 2.
 *   Section 4  LRMSD: centring, R = sum x y^T, the 4x4 matrix T, its largest
 *              eigenpair, U(q), LRMSD = sqrt((sum |x|^2+|y|^2 - 2 lambda)/N).
 *
 * Readings taken where the paper is silent or ambiguous (each one is also
 * listed in the design notes):
 *   - the first transform of a chain, R_0, is the identity (Section 3 says a
 *     residue index j < 0 gives the identity; the peptide bond "of residue
 *     j-1" for j = 0 does not exist), so omega_0 is unused and its gradient 0;
 *   - omega row entry j is the dihedral CA_{j-1} C_{j-1} N_j CA_j, so in the
 *     full-atom graph residue j's R_4 uses omega_{j+1} and places N_{j+1};
 *   - R' is the rotation by 122.686 degrees about x that gives L chirality
 *     at CA; in the paper's R_x convention that is R_x(-122.686 deg);
 *   - the rigid-group geometry (theta_i, d_i, r0) of the side chains is not
 *     printed in the paper; the internal coordinates below are authored from
 *     ideal stereochemistry (bond lengths and angles of Engh & Huber, Acta Cryst.
 *     A47 (1991) 392-400), backbone entries equal the Section 3 constants;
 *     the HIS ring angles at ND1 and CD2 and the proline ring's fixed chi1
 *     and CD dihedral are fitted so that those rings close at the Engh &
 *     Huber closure bond and angles;
 *   - the LRMSD gradient is the exact derivative of the stated LRMSD with
 *     respect to the input y, (y'_i - U x'_i)/(N LRMSD).
 */
#include "tpl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846
#define DEG (PI / 180.0)

/* ------------------------------------------------------------------ */
/* 4x4 homogeneous matrices, row-major double[16]                      */
/* ------------------------------------------------------------------ */

static void mat_identity(double* M) {
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void mat_mul(const double* A, const double* B, double* C) {
    double T[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * r + k] * B[4 * k + c];
            T[4 * r + c] = s;
        }
    memcpy(C, T, sizeof(T));
}

/* y = M (x, 1): position part of M applied to a point. */
static void mat_apply_point(const double* M, const double* x, double* y) {
    double t[3];
    for (int r = 0; r < 3; ++r)
        t[r] = M[4 * r + 0] * x[0] + M[4 * r + 1] * x[1] + M[4 * r + 2] * x[2] + M[4 * r + 3];
    y[0] = t[0]; y[1] = t[1]; y[2] = t[2];
}

/* Inverse of a rigid transform [Q t; 0 1] is [Q^T  -Q^T t; 0 1]. */
static void mat_rigid_inverse(const double* M, double* Mi) {
    double T[16];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T[4 * r + c] = M[4 * c + r];
    for (int r = 0; r < 3; ++r)
        T[4 * r + 3] = -(T[4 * r + 0] * M[3] + T[4 * r + 1] * M[7] + T[4 * r + 2] * M[11]);
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
    memcpy(Mi, T, sizeof(T));
}

/* Section 2: R_x(alpha), R_y(theta), T_x(d) as 4x4 matrices. */
static void mat_rot_x(double a, double* M) {
    mat_identity(M);
    M[5] = cos(a); M[6] = -sin(a);
    M[9] = sin(a); M[10] = cos(a);
}
static void mat_rot_y(double a, double* M) {
    mat_identity(M);
    M[0] = cos(a); M[2] = sin(a);
    M[8] = -sin(a); M[10] = cos(a);
}
static void mat_trans_x(double d, double* M) {
    mat_identity(M);
    M[3] = d;
}

/* Section 3: the explicit matrix R(alpha, theta, d). */
static void mat_R(double alpha, double theta, double d, double* M) {
    double ca = cos(alpha), sa = sin(alpha), ct = cos(theta), st = sin(theta);
    M[0] = ct;  M[1] = sa * st; M[2] = ca * st;  M[3] = d * ct;
    M[4] = 0.0; M[5] = ca;      M[6] = -sa;      M[7] = 0.0;
    M[8] = -st; M[9] = sa * ct; M[10] = ca * ct; M[11] = -d * st;
    M[12] = 0.0; M[13] = 0.0;   M[14] = 0.0;     M[15] = 1.0;
}

/* dR(alpha, theta, d)/dalpha = R_y(theta) T_x(d) dR_x(alpha)/dalpha. */
static void mat_dR(double alpha, double theta, double d, double* M) {
    double Ry[16], Tx[16], dRx[16], T[16];
    mat_rot_y(theta, Ry);
    mat_trans_x(d, Tx);
    memset(dRx, 0, sizeof(dRx));
    dRx[5] = -sin(alpha); dRx[6] = -cos(alpha);
    dRx[9] = cos(alpha);  dRx[10] = -sin(alpha);
    mat_mul(Ry, Tx, T);
    mat_mul(T, dRx, M);
}

/* F = M_parent dR M_node^{-1}; returns F r (3-vector) for a point r. */
static void lever_apply(const double* F, const double* r, double* out) {
    for (int k = 0; k < 3; ++k)
        out[k] = F[4 * k + 0] * r[0] + F[4 * k + 1] * r[1] + F[4 * k + 2] * r[2] + F[4 * k + 3];
}

static void make_lever(const double* M_parent, double alpha, double theta, double d,
                       const double* M_node, double* F) {
    double dR[16], Mi[16], T[16];
    mat_dR(alpha, theta, d, dR);
    mat_rigid_inverse(M_node, Mi);
    mat_mul(M_parent, dR, T);
    mat_mul(T, Mi, F);
}

/* ------------------------------------------------------------------ */
/* Section 3: backbone constants                                      */
/* ------------------------------------------------------------------ */

/* atom i = 3j + k:  k = 0 N (omega_j), 1 CA (phi_j), 2 C (psi_j) */
static const double BB_THETA[3] = {PI - 2.1186, PI - 1.9391, PI - 2.0610};
static const double BB_D[3] = {1.330, 1.460, 1.525};
/* angle row of the transform that places atom k of a residue */
static const int BB_ROW[3] = {2, 0, 1};

static int check_dims(int B, int Lmax) { return (B < 0 || Lmax < 0) ? 1 : 0; }

/* Cumulative transforms M_i = R_0 R_1 ... R_i for one chain, 16 doubles per atom. */
static void backbone_frames(const double* ang, int Lmax, int L, double* M) {
    double cur[16], Ri[16];
    mat_identity(cur);
    for (int j = 0; j < L; ++j)
        for (int k = 0; k < 3; ++k) {
            int i = 3 * j + k;
            if (i == 0) {
                mat_identity(Ri); /* R_0 = I */
            } else {
                double alpha = ang[BB_ROW[k] * Lmax + j];
                mat_R(alpha, BB_THETA[k], BB_D[k], Ri);
            }
            mat_mul(cur, Ri, cur);
            memcpy(M + 16 * i, cur, sizeof(cur));
        }
}

int oracle_backbone_forward(const double* angles, const int32_t* lengths, int B, int Lmax,
                            double* coords) {
    if (check_dims(B, Lmax)) return 1;
    double* M = (double*)malloc((size_t)(3 * (Lmax > 0 ? Lmax : 1)) * 16 * sizeof(double));
    if (!M) return 2;
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        if (L < 0 || L > Lmax) { free(M); return 1; }
        const double* ang = angles + (size_t)b * 3 * Lmax;
        double* out = coords + (size_t)b * 3 * Lmax * 3;
        memset(out, 0, (size_t)3 * Lmax * 3 * sizeof(double));
        backbone_frames(ang, Lmax, L, M);
        for (int i = 0; i < 3 * L; ++i) {
            /* r_i = M_i 0 */
            out[3 * i + 0] = M[16 * i + 3];
            out[3 * i + 1] = M[16 * i + 7];
            out[3 * i + 2] = M[16 * i + 11];
        }
    }
    free(M);
    return 0;
}

int oracle_backbone_backward(const double* angles, const int32_t* lengths, int B, int Lmax,
                             const double* grad_coords, double* grad_angles) {
    if (check_dims(B, Lmax)) return 1;
    double* M = (double*)malloc((size_t)(3 * (Lmax > 0 ? Lmax : 1)) * 16 * sizeof(double));
    if (!M) return 2;
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        if (L < 0 || L > Lmax) { free(M); return 1; }
        const double* ang = angles + (size_t)b * 3 * Lmax;
        const double* g = grad_coords + (size_t)b * 3 * Lmax * 3;
        double* ga = grad_angles + (size_t)b * 3 * Lmax;
        memset(ga, 0, (size_t)3 * Lmax * sizeof(double));
        backbone_frames(ang, Lmax, L, M);
        double I[16];
        mat_identity(I);
        for (int j = 0; j < L; ++j)
            for (int k = 0; k < 3; ++k) {
                int node = 3 * j + k;
                if (node == 0) continue; /* R_0 = I carries no angle */
                double alpha = ang[BB_ROW[k] * Lmax + j];
                const double* Mparent = M + 16 * (node - 1);
                double F[16];
                make_lever(Mparent, alpha, BB_THETA[k], BB_D[k], M + 16 * node, F);
                double s = 0.0;
                for (int i = node; i < 3 * L; ++i) {
                    double r[3] = {M[16 * i + 3], M[16 * i + 7], M[16 * i + 11]};
                    double dr[3];
                    lever_apply(F, r, dr);
                    s += g[3 * i + 0] * dr[0] + g[3 * i + 1] * dr[1] + g[3 * i + 2] * dr[2];
                }
                ga[BB_ROW[k] * Lmax + j] = s;
            }
    }
    free(M);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Section 2: full-atom residue tables (authored internal coordinates) */
/* ------------------------------------------------------------------ */

#define NRES 20    /* amino acids, codes 0..19 */
#define BB_ONLY 20 /* code 20: a residue with its backbone N, CA, C only (the Section 3 model) */
#define NCODES 21
#define MAXSC 10   /* side-chain atoms per residue (TRP) */
#define MAXAT 14   /* heavy atoms per residue (TRP) */
#define MAXGRP 4

/* One side-chain atom in internal coordinates: bonded to `p`, bond angle
 * (q, p, atom), dihedral (r, q, p, atom).  When `chi` is nonzero the dihedral
 * value is an offset added to the group's chi angle (free or fixed). */
typedef struct {
    const char* name;
    int group; /* side-chain group 1..4 */
    const char* p;
    const char* q;
    const char* r;
    double bond, angle_deg, dihedral_deg;
    int chi;
} zatom;

typedef struct {
    const char* three;
    int n_chi;                   /* free chi angles */
    int n_groups;                /* side-chain groups (n_chi, or 1 for ALA/PRO) */
    double fixed_chi_deg[MAXGRP];/* chi value for groups beyond n_chi */
    int n_sc;
    zatom sc[MAXSC];
} residue_def;

/* Group k's origin atom is listed first among the atoms of group k; it is
 * bonded to group k-1's origin (CA for k = 1). */
static const residue_def RES[NRES] = {
    {"ALA", 0, 1, {0.0}, 1, {
        {"CB", 1, "CA", "N", "C", 1.521, 110.4, 0.0, 0}}},
    {"ARG", 4, 4, {0}, 7, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},
        {"CD", 3, "CG", "CB", "CA", 1.520, 111.3, 0.0, 1},
        {"NE", 4, "CD", "CG", "CB", 1.460, 112.0, 0.0, 1},
        {"CZ", 4, "NE", "CD", "CG", 1.329, 124.2, 0.0, 1},
        {"NH1", 4, "CZ", "NE", "CD", 1.326, 120.0, 0.0, 0},
        {"NH2", 4, "CZ", "NE", "CD", 1.326, 120.0, 180.0, 0}}},
    {"ASN", 2, 2, {0}, 4, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.516, 112.6, 0.0, 1},
        {"OD1", 2, "CG", "CB", "CA", 1.231, 120.8, 0.0, 1},
        {"ND2", 2, "CG", "CB", "CA", 1.328, 116.4, 180.0, 1}}},
    {"ASP", 2, 2, {0}, 4, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.516, 112.6, 0.0, 1},
        {"OD1", 2, "CG", "CB", "CA", 1.249, 118.4, 0.0, 1},
        {"OD2", 2, "CG", "CB", "CA", 1.249, 118.4, 180.0, 1}}},
    {"CYS", 1, 1, {0}, 2, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"SG", 1, "CB", "CA", "N", 1.808, 114.4, 0.0, 1}}},
    {"GLN", 3, 3, {0}, 5, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},
        {"CD", 3, "CG", "CB", "CA", 1.516, 112.6, 0.0, 1},
        {"OE1", 3, "CD", "CG", "CB", 1.231, 120.8, 0.0, 1},
        {"NE2", 3, "CD", "CG", "CB", 1.328, 116.4, 180.0, 1}}},
    {"GLU", 3, 3, {0}, 5, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},
        {"CD", 3, "CG", "CB", "CA", 1.516, 112.6, 0.0, 1},
        {"OE1", 3, "CD", "CG", "CB", 1.249, 118.4, 0.0, 1},
        {"OE2", 3, "CD", "CG", "CB", 1.249, 118.4, 180.0, 1}}},
    {"GLY", 0, 0, {0}, 0, {{0}}},
    {"HIS", 2, 2, {0}, 6, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.497, 113.8, 0.0, 1},
        {"ND1", 2, "CG", "CB", "CA", 1.378, 122.7, 0.0, 1},
        {"CD2", 2, "CG", "CB", "CA", 1.354, 131.0, 180.0, 1},
        {"CE1", 2, "ND1", "CG", "CB", 1.345, 106.9, 180.0, 0},
        {"NE2", 2, "CD2", "CG", "CB", 1.382, 109.6, 180.0, 0}}},
    {"ILE", 2, 2, {0}, 4, {
        {"CB", 1, "CA", "N", "C", 1.540, 111.5, 0.0, 0},
        {"CG1", 2, "CB", "CA", "N", 1.530, 110.4, 0.0, 1},
        {"CG2", 1, "CB", "CA", "N", 1.521, 110.5, -122.6, 1},
        {"CD1", 2, "CG1", "CB", "CA", 1.513, 113.8, 0.0, 1}}},
    {"LEU", 2, 2, {0}, 4, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.530, 116.3, 0.0, 1},
        {"CD1", 2, "CG", "CB", "CA", 1.521, 110.7, 0.0, 1},
        {"CD2", 2, "CG", "CB", "CA", 1.521, 110.7, 122.7, 1}}},
    {"LYS", 4, 4, {0}, 5, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},
        {"CD", 3, "CG", "CB", "CA", 1.520, 111.3, 0.0, 1},
        {"CE", 4, "CD", "CG", "CB", 1.520, 111.3, 0.0, 1},
        {"NZ", 4, "CE", "CD", "CG", 1.489, 111.9, 0.0, 1}}},
    {"MET", 3, 3, {0}, 4, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.520, 114.1, 0.0, 1},
        {"SD", 3, "CG", "CB", "CA", 1.803, 112.7, 0.0, 1},
        {"CE", 3, "SD", "CG", "CB", 1.791, 100.9, 0.0, 1}}},
    {"PHE", 2, 2, {0}, 7, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.502, 113.8, 0.0, 1},
        {"CD1", 2, "CG", "CB", "CA", 1.384, 120.7, 0.0, 1},
        {"CD2", 2, "CG", "CB", "CA", 1.384, 120.7, 180.0, 1},
        {"CE1", 2, "CD1", "CG", "CB", 1.382, 120.7, 180.0, 0},
        {"CE2", 2, "CD2", "CG", "CB", 1.382, 120.7, 180.0, 0},
        {"CZ", 2, "CE1", "CD1", "CG", 1.382, 120.0, 0.0, 0}}},
    {"PRO", 0, 1, {-28.0}, 3, {
        {"CB", 1, "CA", "N", "C", 1.530, 103.0, 0.0, 0},
        {"CG", 1, "CB", "CA", "N", 1.492, 104.5, 0.0, 1},
        {"CD", 1, "CG", "CB", "CA", 1.503, 106.1, 33.0, 0}}},
    {"SER", 1, 1, {0}, 2, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"OG", 1, "CB", "CA", "N", 1.417, 111.1, 0.0, 1}}},
    {"THR", 1, 1, {0}, 3, {
        {"CB", 1, "CA", "N", "C", 1.540, 111.5, 0.0, 0},
        {"OG1", 1, "CB", "CA", "N", 1.433, 109.6, 0.0, 1},
        {"CG2", 1, "CB", "CA", "N", 1.521, 110.5, -120.0, 1}}},
    {"TRP", 2, 2, {0}, 10, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.498, 113.6, 0.0, 1},
        {"CD1", 2, "CG", "CB", "CA", 1.365, 126.9, 0.0, 1},
        {"CD2", 2, "CG", "CB", "CA", 1.433, 126.6, 180.0, 1},
        {"NE1", 2, "CD1", "CG", "CB", 1.374, 110.2, 180.0, 0},
        {"CE2", 2, "CD2", "CG", "CB", 1.409, 107.2, 180.0, 0},
        {"CE3", 2, "CD2", "CG", "CB", 1.398, 133.9, 0.0, 0},
        {"CZ2", 2, "CE2", "CD2", "CG", 1.394, 122.4, 180.0, 0},
        {"CZ3", 2, "CE3", "CD2", "CG", 1.382, 118.6, 180.0, 0},
        {"CH2", 2, "CZ2", "CE2", "CD2", 1.368, 117.5, 0.0, 0}}},
    {"TYR", 2, 2, {0}, 8, {
        {"CB", 1, "CA", "N", "C", 1.530, 110.5, 0.0, 0},
        {"CG", 2, "CB", "CA", "N", 1.512, 113.9, 0.0, 1},
        {"CD1", 2, "CG", "CB", "CA", 1.389, 120.8, 0.0, 1},
        {"CD2", 2, "CG", "CB", "CA", 1.389, 120.8, 180.0, 1},
        {"CE1", 2, "CD1", "CG", "CB", 1.382, 121.2, 180.0, 0},
        {"CE2", 2, "CD2", "CG", "CB", 1.382, 121.2, 180.0, 0},
        {"CZ", 2, "CE1", "CD1", "CG", 1.378, 119.6, 0.0, 0},
        {"OH", 2, "CZ", "CE1", "CD1", 1.376, 119.9, 180.0, 0}}},
    {"VAL", 1, 1, {0}, 3, {
        {"CB", 1, "CA", "N", "C", 1.540, 111.5, 0.0, 0},
        {"CG1", 1, "CB", "CA", "N", 1.521, 110.5, 0.0, 1},
        {"CG2", 1, "CB", "CA", "N", 1.521, 110.5, -122.9, 1}}},
};

/* Backbone O in the M_3 frame: bonded to C, angle CA-C-O, dihedral N-CA-C-O = psi + 180. */
static const double O_BOND = 1.231, O_ANGLE_DEG = 120.1, O_DIHEDRAL_OFFSET_DEG = 180.0;
/* R' of Section 2, about x, in the R_x convention of Section 3 (L chirality). */
static const double RPRIME_DEG = -122.686;

/* Expanded per-type table built once from RES. */
typedef struct {
    int n_atoms;
    char names[MAXAT][8];
    int group[MAXAT];          /* 0 M_0, 1 M_1, 2 M_3, 3..6 side-chain group 1..4 */
    double r0[MAXAT][3];       /* standard-frame position in its group's frame */
    double grp_theta[MAXGRP];  /* group k frame: S_k = S_{k-1} R(chi_k, theta_k, d_k) */
    double grp_d[MAXGRP];
} residue_tab;

static residue_tab TAB[NCODES];

/* Code 20 places only the three atoms of the Section 3 backbone, so a chain
 * of such residues is the backbone model and a batch may mix both models. */
static const residue_def RES_BB = {"BB", 0, 0, {0.0}, 0, {{0}}};
static const residue_def* res_def(int code) { return code < NRES ? &RES[code] : &RES_BB; }
static int TAB_READY = 0;

static int sc_index(const residue_def* rd, const char* name) {
    for (int i = 0; i < rd->n_sc; ++i)
        if (strcmp(rd->sc[i].name, name) == 0) return i;
    return -1;
}

/* Place a point by internal coordinates from three reference points a (dihedral
 * reference), b (angle reference) and c (bonded), using the same convention as
 * the paper's R: build the frame at c whose x axis is b->c and whose xz plane
 * holds a on its z < 0 side, then apply R_x(tau) R_y(pi - angle) to (d, 0, 0). */
static void place_internal(const double* a, const double* b, const double* c, double d,
                           double angle, double tau, double* out) {
    double ex[3], v[3], ez[3], ey[3];
    double n = 0.0;
    for (int k = 0; k < 3; ++k) { ex[k] = c[k] - b[k]; n += ex[k] * ex[k]; }
    n = sqrt(n);
    for (int k = 0; k < 3; ++k) ex[k] /= n;
    double proj = 0.0;
    for (int k = 0; k < 3; ++k) { v[k] = a[k] - b[k]; proj += v[k] * ex[k]; }
    n = 0.0;
    for (int k = 0; k < 3; ++k) { v[k] -= proj * ex[k]; n += v[k] * v[k]; }
    n = sqrt(n);
    for (int k = 0; k < 3; ++k) ez[k] = -v[k] / n;
    ey[0] = ez[1] * ex[2] - ez[2] * ex[1];
    ey[1] = ez[2] * ex[0] - ez[0] * ex[2];
    ey[2] = ez[0] * ex[1] - ez[1] * ex[0];
    double th = PI - angle;
    double lx = d * cos(th), ly = d * sin(th) * sin(tau), lz = -d * sin(th) * cos(tau);
    for (int k = 0; k < 3; ++k) out[k] = c[k] + lx * ex[k] + ly * ey[k] + lz * ez[k];
}

/* r0 = R_x(delta) R_y(pi - angle) (d, 0, 0): an atom bonded to a frame's origin
 * whose dihedral is the frame's own rotation angle plus delta. */
static void frame_child(double d, double angle, double delta, double* out) {
    double th = PI - angle;
    out[0] = d * cos(th);
    out[1] = d * sin(th) * sin(delta);
    out[2] = -d * sin(th) * cos(delta);
}

static void build_tables(void) {
    if (TAB_READY) return;
    for (int t = 0; t < NCODES; ++t) {
        const residue_def* rd = res_def(t);
        residue_tab* tb = &TAB[t];
        memset(tb, 0, sizeof(*tb));
        const char* bb[4] = {"N", "CA", "C", "O"};
        for (int k = 0; k < 4; ++k) strcpy(tb->names[k], bb[k]);
        tb->group[0] = 0; tb->group[1] = 1; tb->group[2] = 2; tb->group[3] = 2;
        frame_child(O_BOND, O_ANGLE_DEG * DEG, O_DIHEDRAL_OFFSET_DEG * DEG, tb->r0[3]);
        tb->n_atoms = (t == BB_ONLY) ? 3 : 4 + rd->n_sc; /* no O for the backbone-only code */

        /* Local positions of the atoms of each group in that group's frame. */
        double local[MAXSC][3];
        int have[MAXSC];
        memset(have, 0, sizeof(have));
        /* axis atoms: origin of group k, and origins of k-1, k-2 (CA, N below 1) */
        const char* origin[MAXGRP + 1] = {"CA", 0, 0, 0, 0};
        for (int i = 0; i < rd->n_sc; ++i) {
            const zatom* z = &rd->sc[i];
            if (origin[z->group] == 0) origin[z->group] = z->name;
        }
        for (int k = 1; k <= rd->n_groups; ++k) {
            int oi = sc_index(rd, origin[k]);
            tb->grp_theta[k - 1] = PI - rd->sc[oi].angle_deg * DEG;
            tb->grp_d[k - 1] = rd->sc[oi].bond;
        }
        for (int i = 0; i < rd->n_sc; ++i) {
            const zatom* z = &rd->sc[i];
            int k = z->group;
            const char* prev1 = origin[k - 1];                    /* on the -x axis */
            const char* prev2 = (k >= 2) ? origin[k - 2] : "N";
            double prev1_pos[3] = {-tb->grp_d[k - 1], 0.0, 0.0};
            if (strcmp(z->name, origin[k]) == 0) {
                local[i][0] = local[i][1] = local[i][2] = 0.0;
            } else if (strcmp(z->p, origin[k]) == 0 && strcmp(z->q, prev1) == 0 &&
                       strcmp(z->r, prev2) == 0) {
                /* dihedral (prev2, prev1, origin, atom) = chi_k + offset */
                frame_child(z->bond, z->angle_deg * DEG, z->dihedral_deg * DEG, local[i]);
            } else {
                /* all three references are rigid in this group's frame */
                const char* refs[3] = {z->r, z->q, z->p};
                double pos[3][3];
                for (int m = 0; m < 3; ++m) {
                    if (strcmp(refs[m], prev1) == 0) {
                        memcpy(pos[m], prev1_pos, sizeof(prev1_pos));
                    } else {
                        int ri = sc_index(rd, refs[m]);
                        if (ri < 0 || !have[ri] || rd->sc[ri].group != k) abort();
                        memcpy(pos[m], local[ri], sizeof(pos[m]));
                    }
                }
                place_internal(pos[0], pos[1], pos[2], z->bond, z->angle_deg * DEG,
                               z->dihedral_deg * DEG, local[i]);
            }
            have[i] = 1;
            strcpy(tb->names[4 + i], z->name);
            tb->group[4 + i] = 2 + k;
            memcpy(tb->r0[4 + i], local[i], sizeof(local[i]));
        }
    }
    TAB_READY = 1;
}

int oracle_residue_info(int code, char* three_letter4, int* n_atoms, int* n_chi) {
    if (code < 0 || code >= NCODES) return 1;
    build_tables();
    if (three_letter4) { strncpy(three_letter4, res_def(code)->three, 3); three_letter4[3] = 0; }
    if (n_atoms) *n_atoms = TAB[code].n_atoms;
    if (n_chi) *n_chi = res_def(code)->n_chi;
    return 0;
}

int oracle_residue_atom(int code, int idx, char* name8, int* group) {
    if (code < 0 || code >= NCODES) return 1;
    build_tables();
    if (idx < 0 || idx >= TAB[code].n_atoms) return 1;
    if (name8) strcpy(name8, TAB[code].names[idx]);
    if (group) *group = TAB[code].group[idx];
    return 0;
}

int oracle_residue_atom_r0(int code, int idx, double* r0) {
    if (code < 0 || code >= NCODES) return 1;
    build_tables();
    if (idx < 0 || idx >= TAB[code].n_atoms) return 1;
    memcpy(r0, TAB[code].r0[idx], 3 * sizeof(double));
    return 0;
}

int oracle_fullatom_chain_atoms(const uint8_t* seq, int length) {
    build_tables();
    int n = 0;
    for (int j = 0; j < length; ++j) {
        if (seq[j] >= NCODES) return -1;
        n += TAB[seq[j]].n_atoms;
    }
    return n;
}

/* Per-residue frames of the full-atom graph. */
typedef struct {
    double M0[16];  /* frame of N_j (previous residue's M_4, identity for j = 0) */
    double M1[16];  /* M_0 R_1(phi) */
    double M3[16];  /* M_1 R_3(psi) */
    double S0[16];  /* M_1 R' */
    double S[MAXGRP][16]; /* side-chain group frames */
} residue_frames;

static double chi_value(const double* ang, int Lmax, int j, const residue_def* rd, int k) {
    /* group k (1-based) uses chi_k when free, else the table's fixed value */
    if (k <= rd->n_chi) return ang[(3 + k - 1) * Lmax + j];
    return rd->fixed_chi_deg[k - 1] * DEG;
}

static void fullatom_frames(const double* ang, const uint8_t* seq, int Lmax, int L,
                            residue_frames* F) {
    double cur[16], T[16], Rp[16];
    mat_identity(cur);
    mat_rot_x(RPRIME_DEG * DEG, Rp);
    for (int j = 0; j < L; ++j) {
        const residue_def* rd = res_def(seq[j]);
        const residue_tab* tb = &TAB[seq[j]];
        residue_frames* f = &F[j];
        memcpy(f->M0, cur, sizeof(cur));
        mat_R(ang[0 * Lmax + j], BB_THETA[1], BB_D[1], T);
        mat_mul(f->M0, T, f->M1);
        mat_R(ang[1 * Lmax + j], BB_THETA[2], BB_D[2], T);
        mat_mul(f->M1, T, f->M3);
        mat_mul(f->M1, Rp, f->S0);
        const double* parent = f->S0;
        for (int k = 1; k <= rd->n_groups; ++k) {
            mat_R(chi_value(ang, Lmax, j, rd, k), tb->grp_theta[k - 1], tb->grp_d[k - 1], T);
            mat_mul(parent, T, f->S[k - 1]);
            parent = f->S[k - 1];
        }
        if (j + 1 < L) {
            /* M_4 = M_3 R_4(omega_{j+1}) places N_{j+1} */
            mat_R(ang[2 * Lmax + j + 1], BB_THETA[0], BB_D[0], T);
            mat_mul(f->M3, T, cur);
        }
    }
}

static const double* group_frame(const residue_frames* f, int g) {
    switch (g) {
        case 0: return f->M0;
        case 1: return f->M1;
        case 2: return f->M3;
        default: return f->S[g - 3];
    }
}

static int check_seq(const uint8_t* seq, int L) {
    for (int j = 0; j < L; ++j)
        if (seq[j] >= NCODES) return 1;
    return 0;
}

int oracle_fullatom_forward(const double* angles, const uint8_t* seq, const int32_t* lengths,
                            int B, int Lmax, int Amax, double* coords, int32_t* num_atoms) {
    if (check_dims(B, Lmax) || Amax < 0) return 1;
    build_tables();
    residue_frames* F = (residue_frames*)malloc((size_t)(Lmax > 0 ? Lmax : 1) * sizeof(residue_frames));
    if (!F) return 2;
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        const uint8_t* s = seq + (size_t)b * Lmax;
        if (L < 0 || L > Lmax || check_seq(s, L)) { free(F); return 1; }
        int na = oracle_fullatom_chain_atoms(s, L);
        if (na > Amax) { free(F); return 1; }
        const double* ang = angles + (size_t)b * 7 * Lmax;
        double* out = coords + (size_t)b * Amax * 3;
        memset(out, 0, (size_t)Amax * 3 * sizeof(double));
        fullatom_frames(ang, s, Lmax, L, F);
        int a = 0;
        for (int j = 0; j < L; ++j) {
            const residue_tab* tb = &TAB[s[j]];
            for (int t = 0; t < tb->n_atoms; ++t, ++a)
                mat_apply_point(group_frame(&F[j], tb->group[t]), tb->r0[t], out + 3 * a);
        }
        num_atoms[b] = na;
    }
    free(F);
    return 0;
}

int oracle_fullatom_backward(const double* angles, const uint8_t* seq, const int32_t* lengths,
                             int B, int Lmax, int Amax, const double* grad_coords,
                             double* grad_angles) {
    if (check_dims(B, Lmax) || Amax < 0) return 1;
    build_tables();
    residue_frames* F = (residue_frames*)malloc((size_t)(Lmax > 0 ? Lmax : 1) * sizeof(residue_frames));
    int* off = (int*)malloc((size_t)(Lmax + 1) * sizeof(int));
    double* r = (double*)malloc((size_t)(Amax > 0 ? Amax : 1) * 3 * sizeof(double));
    if (!F || !off || !r) { free(F); free(off); free(r); return 2; }
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        const uint8_t* s = seq + (size_t)b * Lmax;
        if (L < 0 || L > Lmax || check_seq(s, L)) { free(F); free(off); free(r); return 1; }
        int na = oracle_fullatom_chain_atoms(s, L);
        if (na > Amax) { free(F); free(off); free(r); return 1; }
        const double* ang = angles + (size_t)b * 7 * Lmax;
        const double* g = grad_coords + (size_t)b * Amax * 3;
        double* ga = grad_angles + (size_t)b * 7 * Lmax;
        memset(ga, 0, (size_t)7 * Lmax * sizeof(double));
        fullatom_frames(ang, s, Lmax, L, F);
        off[0] = 0;
        for (int j = 0; j < L; ++j) {
            const residue_tab* tb = &TAB[s[j]];
            for (int t = 0; t < tb->n_atoms; ++t)
                mat_apply_point(group_frame(&F[j], tb->group[t]), tb->r0[t], r + 3 * (off[j] + t));
            off[j + 1] = off[j] + tb->n_atoms;
        }
        for (int j = 0; j < L; ++j) {
            const residue_def* rd = res_def(s[j]);
            const residue_tab* tb = &TAB[s[j]];
            double Fm[16], dr[3];
            /* phi_j: node M_1 = M_0 R_1(phi); children: every atom of residue j but N,
             * and all later residues. */
            {
                make_lever(F[j].M0, ang[0 * Lmax + j], BB_THETA[1], BB_D[1], F[j].M1, Fm);
                double acc = 0.0;
                for (int a = off[j] + 1; a < na; ++a) {
                    lever_apply(Fm, r + 3 * a, dr);
                    acc += g[3 * a] * dr[0] + g[3 * a + 1] * dr[1] + g[3 * a + 2] * dr[2];
                }
                ga[0 * Lmax + j] = acc;
            }
            /* psi_j: node M_3 = M_1 R_3(psi); children: C, O of residue j and all later
             * residues. */
            {
                make_lever(F[j].M1, ang[1 * Lmax + j], BB_THETA[2], BB_D[2], F[j].M3, Fm);
                double acc = 0.0;
                for (int t = 0; t < tb->n_atoms; ++t) {
                    if (tb->group[t] != 2) continue;
                    int a = off[j] + t;
                    lever_apply(Fm, r + 3 * a, dr);
                    acc += g[3 * a] * dr[0] + g[3 * a + 1] * dr[1] + g[3 * a + 2] * dr[2];
                }
                for (int a = off[j + 1]; a < na; ++a) {
                    lever_apply(Fm, r + 3 * a, dr);
                    acc += g[3 * a] * dr[0] + g[3 * a + 1] * dr[1] + g[3 * a + 2] * dr[2];
                }
                ga[1 * Lmax + j] = acc;
            }
            /* omega_j (j >= 1): node M_0 of residue j = M_3(j-1) R_4(omega_j); children:
             * every atom of residues j.. */
            if (j >= 1) {
                make_lever(F[j - 1].M3, ang[2 * Lmax + j], BB_THETA[0], BB_D[0], F[j].M0, Fm);
                double acc = 0.0;
                for (int a = off[j]; a < na; ++a) {
                    lever_apply(Fm, r + 3 * a, dr);
                    acc += g[3 * a] * dr[0] + g[3 * a + 1] * dr[1] + g[3 * a + 2] * dr[2];
                }
                ga[2 * Lmax + j] = acc;
            }
            /* chi_k: node S_k = S_{k-1} R(chi_k); children: atoms of groups k.. */
            for (int k = 1; k <= rd->n_chi; ++k) {
                const double* parent = (k == 1) ? F[j].S0 : F[j].S[k - 2];
                make_lever(parent, ang[(3 + k - 1) * Lmax + j], tb->grp_theta[k - 1],
                           tb->grp_d[k - 1], F[j].S[k - 1], Fm);
                double acc = 0.0;
                for (int t = 0; t < tb->n_atoms; ++t) {
                    if (tb->group[t] < 2 + k) continue;
                    int a = off[j] + t;
                    lever_apply(Fm, r + 3 * a, dr);
                    acc += g[3 * a] * dr[0] + g[3 * a + 1] * dr[1] + g[3 * a + 2] * dr[2];
                }
                ga[(3 + k - 1) * Lmax + j] = acc;
            }
        }
    }
    free(F); free(off); free(r);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Section 3 backbone with the carbonyl O of each residue              */
/* ------------------------------------------------------------------ */

/* The paper's backbone model places N, CA and C only.  The carbonyl O of
 * residue j is rigid in the frame M_{3j+2} of C_j (after the psi_j rotation),
 * where the full-atom residue tables put it: bond C-O, angle CA-C-O,
 * dihedral N-CA-C-O = psi_j + 180 (so it lies in the plane of CA_j, C_j and
 * N_{j+1}, opposite N_{j+1}): O_j = M_{3j+2} r0_O. */
static void backbone_o_local(double* r0) {
    frame_child(O_BOND, O_ANGLE_DEG * DEG, O_DIHEDRAL_OFFSET_DEG * DEG, r0);
}

int oracle_backbone_forward_o(const double* angles, const int32_t* lengths, int B, int Lmax,
                              double* coords, double* o_coords) {
    if (oracle_backbone_forward(angles, lengths, B, Lmax, coords)) return 1;
    double* M = (double*)malloc((size_t)(3 * (Lmax > 0 ? Lmax : 1)) * 16 * sizeof(double));
    if (!M) return 2;
    double r0[3];
    backbone_o_local(r0);
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        double* o = o_coords + (size_t)b * Lmax * 3;
        memset(o, 0, (size_t)Lmax * 3 * sizeof(double));
        backbone_frames(angles + (size_t)b * 3 * Lmax, Lmax, L, M);
        for (int j = 0; j < L; ++j) mat_apply_point(M + 16 * (3 * j + 2), r0, o + 3 * j);
    }
    free(M);
    return 0;
}

/* Eq. 2 with the O atoms among the moved atoms: O_j moves with every angle of
 * the nodes 0 .. 3j+2 (up to and including psi_j). */
int oracle_backbone_backward_o(const double* angles, const int32_t* lengths, int B, int Lmax,
                               const double* grad_coords, const double* grad_o, double* grad_angles) {
    if (check_dims(B, Lmax)) return 1;
    double* M = (double*)malloc((size_t)(3 * (Lmax > 0 ? Lmax : 1)) * 16 * sizeof(double));
    double* O = (double*)malloc((size_t)(Lmax > 0 ? Lmax : 1) * 3 * sizeof(double));
    if (!M || !O) { free(M); free(O); return 2; }
    double r0[3];
    backbone_o_local(r0);
    for (int b = 0; b < B; ++b) {
        int L = lengths[b];
        if (L < 0 || L > Lmax) { free(M); free(O); return 1; }
        const double* ang = angles + (size_t)b * 3 * Lmax;
        const double* g = grad_coords + (size_t)b * 3 * Lmax * 3;
        const double* go = grad_o + (size_t)b * Lmax * 3;
        double* ga = grad_angles + (size_t)b * 3 * Lmax;
        memset(ga, 0, (size_t)3 * Lmax * sizeof(double));
        backbone_frames(ang, Lmax, L, M);
        for (int j = 0; j < L; ++j) mat_apply_point(M + 16 * (3 * j + 2), r0, O + 3 * j);
        for (int j = 0; j < L; ++j)
            for (int k = 0; k < 3; ++k) {
                int node = 3 * j + k;
                if (node == 0) continue; /* R_0 = I carries no angle */
                double alpha = ang[BB_ROW[k] * Lmax + j];
                double F[16], dr[3];
                make_lever(M + 16 * (node - 1), alpha, BB_THETA[k], BB_D[k], M + 16 * node, F);
                double s = 0.0;
                for (int i = node; i < 3 * L; ++i) {
                    double r[3] = {M[16 * i + 3], M[16 * i + 7], M[16 * i + 11]};
                    lever_apply(F, r, dr);
                    s += g[3 * i + 0] * dr[0] + g[3 * i + 1] * dr[1] + g[3 * i + 2] * dr[2];
                }
                for (int jo = 0; jo < L; ++jo) {
                    if (3 * jo + 2 < node) continue;
                    lever_apply(F, O + 3 * jo, dr);
                    s += go[3 * jo + 0] * dr[0] + go[3 * jo + 1] * dr[1] + go[3 * jo + 2] * dr[2];
                }
                ga[BB_ROW[k] * Lmax + j] = s;
            }
    }
    free(M);
    free(O);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Section 4: LRMSD                                                    */
/* ------------------------------------------------------------------ */

/* Cyclic Jacobi for a real symmetric 4x4 (textbook method): repeated plane
 * rotations that zero one off-diagonal entry at a time. */
int oracle_sym4_eig(const double* A_in, double* evals, double* evecs) {
    double A[16], V[16];
    memcpy(A, A_in, sizeof(A));
    mat_identity(V);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) {
                tot += A[4 * p + q] * A[4 * p + q];
                if (p != q) off += A[4 * p + q] * A[4 * p + q];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < 3; ++p)
            for (int q = p + 1; q < 4; ++q) {
                double apq = A[4 * p + q];
                if (apq == 0.0) continue;
                double theta = (A[4 * q + q] - A[4 * p + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J, V <- V J with J the (p,q) rotation */
                for (int k = 0; k < 4; ++k) {
                    double akp = A[4 * k + p], akq = A[4 * k + q];
                    A[4 * k + p] = c * akp - s * akq;
                    A[4 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {
                    double apk = A[4 * p + k], aqk = A[4 * q + k];
                    A[4 * p + k] = c * apk - s * aqk;
                    A[4 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[4 * k + p], vkq = V[4 * k + q];
                    V[4 * k + p] = c * vkp - s * vkq;
                    V[4 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    /* sort ascending */
    int idx[4] = {0, 1, 2, 3};
    for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
            if (A[5 * idx[b]] < A[5 * idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    for (int a = 0; a < 4; ++a) {
        evals[a] = A[5 * idx[a]];
        for (int k = 0; k < 4; ++k) evecs[4 * k + a] = V[4 * k + idx[a]];
    }
    return 0;
}

typedef struct {
    int n;
    double xc[3], yc[3]; /* centroids of target x and input y */
    double U[9];
    double lambda, e0, lrmsd;
} lrmsd_state;

static void lrmsd_one(const double* y, const double* x, int n, lrmsd_state* st) {
    memset(st, 0, sizeof(*st));
    st->n = n;
    if (n <= 0) return;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) { st->xc[k] += x[3 * i + k]; st->yc[k] += y[3 * i + k]; }
    for (int k = 0; k < 3; ++k) { st->xc[k] /= n; st->yc[k] /= n; }
    /* R = sum x_i y_i^T on centred coordinates; E0 = sum |x|^2 + |y|^2 */
    double R[3][3] = {{0}};
    double e0 = 0.0;
    for (int i = 0; i < n; ++i) {
        double xi[3], yi[3];
        for (int k = 0; k < 3; ++k) { xi[k] = x[3 * i + k] - st->xc[k]; yi[k] = y[3 * i + k] - st->yc[k]; }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) R[a][b] += xi[a] * yi[b];
        e0 += xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2] + yi[0] * yi[0] + yi[1] * yi[1] + yi[2] * yi[2];
    }
    /* T(R), 1-based R_ab of the paper mapped to R[a-1][b-1] */
    double T[16] = {
        R[0][0] + R[1][1] + R[2][2], R[1][2] - R[2][1], R[2][0] - R[0][2], R[0][1] - R[1][0],
        R[1][2] - R[2][1], R[0][0] - R[1][1] - R[2][2], R[0][1] + R[1][0], R[0][2] + R[2][0],
        R[2][0] - R[0][2], R[0][1] + R[1][0], -R[0][0] + R[1][1] - R[2][2], R[1][2] + R[2][1],
        R[0][1] - R[1][0], R[0][2] + R[2][0], R[1][2] + R[2][1], -R[0][0] - R[1][1] + R[2][2]};
    double ev[4], V[16];
    oracle_sym4_eig(T, ev, V);
    double q[4] = {V[0 * 4 + 3], V[1 * 4 + 3], V[2 * 4 + 3], V[3 * 4 + 3]};
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) q[k] /= qn;
    double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    double* U = st->U;
    U[0] = q0 * q0 + q1 * q1 - q2 * q2 - q3 * q3; U[1] = 2 * (q1 * q2 - q0 * q3); U[2] = 2 * (q1 * q3 + q0 * q2);
    U[3] = 2 * (q1 * q2 + q0 * q3); U[4] = q0 * q0 - q1 * q1 + q2 * q2 - q3 * q3; U[5] = 2 * (q2 * q3 - q0 * q1);
    U[6] = 2 * (q1 * q3 - q0 * q2); U[7] = 2 * (q2 * q3 + q0 * q1); U[8] = q0 * q0 - q1 * q1 - q2 * q2 + q3 * q3;
    st->lambda = ev[3];
    st->e0 = e0;
    double rad = (e0 - 2.0 * ev[3]) / n;
    st->lrmsd = sqrt(rad > 0.0 ? rad : 0.0);
}

int oracle_lrmsd_forward(const double* input, const double* target, const int32_t* num_atoms,
                         int P, int Nmax, double* lrmsd, double* U_out, double* lambda_out) {
    if (P < 0 || Nmax < 0) return 1;
    for (int p = 0; p < P; ++p) {
        int n = num_atoms[p];
        if (n < 0 || n > Nmax) return 1;
        lrmsd_state st;
        lrmsd_one(input + (size_t)p * Nmax * 3, target + (size_t)p * Nmax * 3, n, &st);
        lrmsd[p] = st.lrmsd;
        if (U_out) memcpy(U_out + 9 * (size_t)p, st.U, sizeof(st.U));
        if (lambda_out) lambda_out[p] = st.lambda;
    }
    return 0;
}

int oracle_lrmsd_backward(const double* grad_lrmsd, const double* input, const double* target,
                          const int32_t* num_atoms, int P, int Nmax, double* grad_input) {
    if (P < 0 || Nmax < 0) return 1;
    for (int p = 0; p < P; ++p) {
        int n = num_atoms[p];
        if (n < 0 || n > Nmax) return 1;
        const double* y = input + (size_t)p * Nmax * 3;
        const double* x = target + (size_t)p * Nmax * 3;
        double* gy = grad_input + (size_t)p * Nmax * 3;
        memset(gy, 0, (size_t)Nmax * 3 * sizeof(double));
        lrmsd_state st;
        lrmsd_one(y, x, n, &st);
        if (n == 0 || st.lrmsd < 1e-12) continue;
        double scale = grad_lrmsd[p] / (n * st.lrmsd);
        for (int i = 0; i < n; ++i) {
            double xi[3], yi[3];
            for (int k = 0; k < 3; ++k) { xi[k] = x[3 * i + k] - st.xc[k]; yi[k] = y[3 * i + k] - st.yc[k]; }
            for (int a = 0; a < 3; ++a) {
                double ux = st.U[3 * a] * xi[0] + st.U[3 * a + 1] * xi[1] + st.U[3 * a + 2] * xi[2];
                gy[3 * i + a] = scale * (yi[a] - ux);
            }
        }
    }
    return 0;
}
