/*
 * Plain FP64 CPU oracle for the angles -> coordinates mapping (backbone and
 * full-atom), its adjoint, and LRMSD, written from the paper
 * "TorchProteinLibrary: A computationally efficient, differentiable
 * representation of protein structure" (Derevyanko & Lamoureux, 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two agree only because both
 * follow the paper.
 *
 * Layouts (all row-major, caller-owned host memory, FP64):
 *   backbone angles   [B][3][Lmax]  rows phi, psi, omega
 *   backbone coords   [B][3*Lmax][3] atoms N, CA, C per residue
 *   full-atom angles  [B][7][Lmax]  rows phi, psi, omega, chi1..chi4
 *   full-atom coords  [B][Amax][3]
 *   sequences         [B][Lmax] uint8 residue codes 0..19 (ALA ARG ASN ASP
 *                     CYS GLN GLU GLY HIS ILE LEU LYS MET PHE PRO SER THR TRP
 *                     TYR VAL) and 20 = backbone only (N, CA, C: the Section 3
 *                     model), so one batch may mix both models
 *   LRMSD clouds      [P][Nmax][3]
 * Padding (residue >= length, atom >= num_atoms) is ignored on input and
 * written as 0 on output.  Functions return 0 on success, nonzero on a bad
 * argument (no partial outputs are promised in that case).
 */
#ifndef TPL_ORACLE_H
#define TPL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Section 3: r_i = R_0 R_1 ... R_i 0 with the per-atom constants of the
 * backbone itemization.  R_0 is the identity (first transform of the chain). */
int oracle_backbone_forward(const double* angles, const int32_t* lengths,
                            int B, int Lmax, double* coords);

/* Section 3, Eq. 2: dL/dalpha_k = sum_{i>=k} g_i . (M_{k-1} dR_k/dalpha M_k^{-1} r_i).
 * O(L^2) per chain, exactly as the sums are written. */
int oracle_backbone_backward(const double* angles, const int32_t* lengths,
                             int B, int Lmax, const double* grad_coords,
                             double* grad_angles);

/* Section 3 with the carbonyl O of each residue (not placed by the paper's
 * backbone model): O_j rigid in the frame of C_j after psi_j, bond C-O, angle
 * CA-C-O and dihedral N-CA-C-O = psi_j + 180 as in the full-atom tables.
 * coords as oracle_backbone_forward; o_coords [B][Lmax][3]. */
int oracle_backbone_forward_o(const double* angles, const int32_t* lengths, int B, int Lmax,
                              double* coords, double* o_coords);

/* Eq. 2 with the O atoms moved by every angle up to their residue's psi:
 * grad_coords [B][3*Lmax][3], grad_o [B][Lmax][3]. */
int oracle_backbone_backward_o(const double* angles, const int32_t* lengths, int B, int Lmax,
                               const double* grad_coords, const double* grad_o, double* grad_angles);

/* Section 2: graph of cumulative transforms M_1 = M_0 R_1(phi),
 * side-chain frames M_0 R_1 R' R(chi1) ..., M_3 = M_1 R_3(psi),
 * next M_0 = M_3 R_4(omega); atoms r = M_g r0. */
int oracle_fullatom_forward(const double* angles, const uint8_t* seq,
                            const int32_t* lengths, int B, int Lmax, int Amax,
                            double* coords, int32_t* num_atoms);

/* Section 2, Eq. 1: dL/dalpha_i = sum_{k in children(i)} g_k . (F_i r_k),
 * F_i = M_parent(i) dR_i/dalpha M_i^{-1}. O(L^2) per chain. */
int oracle_fullatom_backward(const double* angles, const uint8_t* seq,
                             const int32_t* lengths, int B, int Lmax, int Amax,
                             const double* grad_coords, double* grad_angles);

/* Number of heavy atoms of one chain (sum over its residues). -1 on a bad code. */
int oracle_fullatom_chain_atoms(const uint8_t* seq, int length);

/* Residue table queries (for bit-exact comparison with the CUDA library). */
int oracle_residue_info(int code, char* three_letter4, int* n_atoms, int* n_chi);
/* Name of atom `idx` of residue `code`, and its rigid-group index:
 * 0 = M_0 (N), 1 = M_1 (CA), 2 = M_3 (C, O), 3..6 = side-chain groups 1..4. */
int oracle_residue_atom(int code, int idx, char* name8, int* group);
/* Standard-frame position r0 of atom `idx` of residue `code` (3 doubles). */
int oracle_residue_atom_r0(int code, int idx, double* r0);

/* Section 4: LRMSD(x = target, y = input) by the Coutsias-Seok-Dill quaternion
 * method: centre, R = sum x y^T, T(R), largest eigenpair of T by cyclic Jacobi,
 * U(q), LRMSD = sqrt((sum |x|^2 + |y|^2 - 2 lambda) / N).  Optional outputs
 * (may be NULL): U [P][9] row-major, lambda [P]. */
int oracle_lrmsd_forward(const double* input, const double* target,
                         const int32_t* num_atoms, int P, int Nmax,
                         double* lrmsd, double* U_out, double* lambda_out);

/* Gradient of LRMSD with respect to the input coordinates y:
 * dLRMSD/dy_i = (y'_i - U x'_i) / (N LRMSD), scaled by grad_lrmsd[p];
 * zero when LRMSD < 1e-12. */
int oracle_lrmsd_backward(const double* grad_lrmsd, const double* input,
                          const double* target, const int32_t* num_atoms,
                          int P, int Nmax, double* grad_input);

/* Symmetric 4x4 eigen-decomposition by cyclic Jacobi (exposed for pins).
 * A row-major [16] (not modified); evals[4] ascending; evecs [16] columns. */
int oracle_sym4_eig(const double* A, double* evals, double* evecs);

#ifdef __cplusplus
}
#endif
#endif
