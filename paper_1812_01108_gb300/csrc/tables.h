// Residue geometry tables of the full-atom model (paper Section 2), built on
// the host from authored internal coordinates and handed to the kernels by
// value (kernel parameter space), so no device-side initialisation is needed.
#pragma once

#include <stdint.h>

namespace tpl {

constexpr int kNumAminoAcids = 20;  // residue codes 0..19
constexpr int kBackboneCode = 20;   // residue code 20: N, CA, C only (the Section 3 backbone)
constexpr int kNumTypes = 21;
constexpr int kMaxAtoms = 14;    // heavy atoms per residue (TRP)
constexpr int kMaxSide = 10;     // side-chain atoms per residue (TRP)
constexpr int kMaxGroups = 4;    // side-chain rigid groups (chi1..chi4)
constexpr int kGlyCode = 7;

// Backbone constants of Section 3: transform k = 0 (N, omega), 1 (CA, phi),
// 2 (C, psi) is R(angle, theta_k, d_k).
struct BackboneConst {
    float ct[3], st[3], d[3];
    float o[3];  // carbonyl O in the frame of C after psi (the full-atom tables' O)
};
struct BackboneConstD {
    double ct[3], st[3], d[3];
    double o[3];
};

// FP32 table for the scan kernels.  Side-chain atoms are listed by group
// (group k's atoms are [grp_end[k-1], grp_end[k])) with their output index.
struct FaTable {
    float4 grp[kNumTypes][kMaxGroups];     // cos theta, sin theta, d, 0
    float2 fixchi[kNumTypes][kMaxGroups];  // cos, sin of the fixed chi of a non-free group
    float4 side[kNumTypes][kMaxSide];      // r0.x, r0.y, r0.z, (output index + 16 * group) as float
    uint8_t n_atoms[kNumTypes];
    uint8_t n_chi[kNumTypes];
    uint8_t n_groups[kNumTypes];
    uint8_t grp_end[kNumTypes][kMaxGroups];
    uint8_t atom_grp[kNumTypes][16];       // rigid group of each output atom (0 M_0, 1 M_1, 2 M_3, 3.. side)
    uint8_t origin[kNumTypes][kMaxGroups]; // output index of side group k's origin atom
    float4 o_r0;        // backbone O in the M_3 frame
    float rp_c, rp_s;   // R' = R_x(rho)
    BackboneConst bb;
};

// FP64 table for the plain per-chain forms: r0 per output atom, its group,
// and the origin atom of each group (the axis of chi_k runs from the origin of
// group k-1, CA for k = 1, to the origin of group k).
struct FaTableD {
    double r0[kNumTypes][kMaxAtoms][3];
    uint8_t group[kNumTypes][kMaxAtoms];  // 0 M_0, 1 M_1, 2 M_3, 3..6 side groups 1..4
    uint8_t origin[kNumTypes][kMaxGroups];
    double grp_ct[kNumTypes][kMaxGroups], grp_st[kNumTypes][kMaxGroups], grp_d[kNumTypes][kMaxGroups];
    double fixchi[kNumTypes][kMaxGroups];
    uint8_t n_atoms[kNumTypes];
    uint8_t n_chi[kNumTypes];
    uint8_t n_groups[kNumTypes];
    double rp_c, rp_s;
    BackboneConstD bb;
};

const FaTable& fa_table();
const FaTableD& fa_table_d();
BackboneConst backbone_const();
BackboneConstD backbone_const_d();

// Host-side metadata for tpl_residue_table / tpl_residue_atom.
const char* residue_three(int code);
const char* residue_atom_name(int code, int idx);

}  // namespace tpl
