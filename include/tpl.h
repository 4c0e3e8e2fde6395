/*
 * tpl.h -- C ABI of the GB300 (sm_103a) library for the differentiable
 * dihedral-angle -> Cartesian-coordinate mapping of proteins and the LRMSD
 * distance, after Derevyanko & Lamoureux, "TorchProteinLibrary: A
 * computationally efficient, differentiable representation of protein
 * structure" (2018).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every tensor pointer is DEVICE memory owned by the caller.  The library
 *    allocates nothing: scratch space is the caller's `workspace`, sized by the
 *    matching *_workspace_size() query.
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream), performs no host synchronisation and no
 *    allocation, and may be captured in a CUDA graph.
 *  - Errors the host can see (bad sizes, NULL pointers, misalignment, short
 *    workspace) are returned at once and nothing is launched.  Errors that
 *    depend on device data (a residue code > 20, a length outside [0, Lmax],
 *    a chain with more atoms than Amax) set bits of a per-device status word
 *    that tpl_get_status() reads and clears; outputs of the affected chain are
 *    then unspecified but no access leaves the caller's buffers.
 *  - Floating tensors are contiguous, row-major, 4-byte aligned; the hot-path
 *    entry points require 16-byte aligned base pointers and Lmax, Amax, Nmax
 *    multiples of 4 (TPL_ERR_MISALIGNED / TPL_ERR_BAD_SHAPE otherwise).
 *  - Padding (residue >= length, atom >= num_atoms) is ignored on input and
 *    written as 0 on output; with TPL_FLAG_PADDING_ZEROED in the options the
 *    chain calls may leave output padding unwritten (the caller keeps it 0).
 *
 * Layouts
 *  - backbone angles  [B][3][Lmax]  rows phi, psi, omega (radians)
 *  - backbone coords  [B][3*Lmax][3] atoms N, CA, C of each residue (Angstrom)
 *  - full-atom angles [B][7][Lmax]  rows phi, psi, omega, chi1, chi2, chi3, chi4
 *  - sequence         [B][Lmax] uint8 residue codes 0..19 = ALA ARG ASN ASP CYS
 *                     GLN GLU GLY HIS ILE LEU LYS MET PHE PRO SER THR TRP TYR VAL;
 *                     20 = BB, a residue with the Section 3 backbone N, CA, C
 *                     only (no O, no side chain): a chain of BB residues is the
 *                     backbone model, so one full-atom call runs a batch that
 *                     mixes both models (chain by chain or residue by residue)
 *  - full-atom coords [B][Amax][3] heavy atoms, residue by residue, each residue
 *                     N, CA, C, O then its side chain (tpl_residue_atom order)
 *  - LRMSD clouds     [P][Nmax][3]
 *
 * Readings of the paper this library implements
 *  - the first transform of a chain is the identity (R_0 = I; Section 3 gives
 *    the identity for a residue index j < 0), so omega_0 is ignored and its
 *    gradient is 0;
 *  - omega entry j is the dihedral CA(j-1) C(j-1) N(j) CA(j): the transform
 *    placing N of residue j (Section 3 itemization);
 *  - R' (Section 2) is the 122.686 degree rotation about x that gives L
 *    chirality at CA;
 *  - side-chain rigid-group geometry (not printed in the paper) comes from an
 *    authored table of ideal internal coordinates;
 *  - the LRMSD gradient is the exact derivative of the stated LRMSD with
 *    respect to the INPUT structure y: (y'_i - U x'_i) / (N LRMSD).
 */
#ifndef TPL_H
#define TPL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int tpl_status;
#define TPL_OK 0
#define TPL_ERR_INVALID_ARG 1      /* NULL pointer, negative size, bad option value */
#define TPL_ERR_BAD_SHAPE 2        /* Lmax / Amax / Nmax not a multiple of 4, or too large */
#define TPL_ERR_MISALIGNED 3       /* a base pointer is not 16-byte aligned */
#define TPL_ERR_WORKSPACE 4        /* workspace NULL or smaller than the size query */
#define TPL_ERR_CUDA 5             /* a CUDA runtime call failed (see tpl_last_error) */
#define TPL_ERR_NO_DEVICE 6        /* no usable CUDA device */

/* Bits of the device status word (tpl_get_status). */
#define TPL_STATUS_BAD_RESIDUE 0x1 /* a residue code > 20 was read */
#define TPL_STATUS_BAD_LENGTH 0x2  /* a length < 0 or > Lmax, or num_atoms outside [0, Nmax] */
#define TPL_STATUS_TOO_MANY_ATOMS 0x4 /* a chain needs more than Amax atoms */
#define TPL_STATUS_ZERO_LRMSD 0x8  /* an LRMSD below 1e-12 A: its gradient is set to 0 */
#define TPL_STATUS_TIMEOUT 0x10    /* a bounded wait between CTAs gave up (results invalid) */
#define TPL_STATUS_BAD_WORKSPACE 0x20 /* a backward was given a workspace its forward did not fill */

typedef struct CUstream_st* tpl_stream; /* same type as cudaStream_t */

#define TPL_BWD_AUTO 0
#define TPL_BWD_RECOMPUTE 1   /* rebuild frames from the angles (fewest HBM bytes) */
#define TPL_BWD_FROM_COORDS 2 /* read the forward's coordinates instead */

#define TPL_SCHED_AUTO 0          /* backbone: PACKED; full atom: BATCH_ORDER */
#define TPL_SCHED_LONGEST_FIRST 1 /* chains sorted by length, longest first */
#define TPL_SCHED_BATCH_ORDER 2   /* chains in batch order */
#define TPL_SCHED_PACKED 3        /* longest first, and chains of at most one tile packed
                                     up to 8 per tile (chains per CTA > 1).  Full atom:
                                     the backward must read the coordinates (a packed
                                     forward with TPL_BWD_RECOMPUTE is rejected; a
                                     backward that rebuilds frames on a packed workspace
                                     sets TPL_STATUS_BAD_WORKSPACE and writes zeros for
                                     those chains); the two-call training step treats
                                     it as LONGEST_FIRST */

/* Launch options; a NULL pointer means all zeros (everything automatic). */
/* tpl_opts.flags */
#define TPL_FLAG_PADDING_ZEROED 0x1 /* the caller keeps the padding of the outputs zero (it zeroed
                                       them once): the chain calls need not write it again */

typedef struct tpl_opts {
    int bwd_mode;       /* TPL_BWD_* */
    int threads;        /* threads per CTA of the chain kernels, 0 = tuned default */
    int res_per_thread; /* consecutive residues per thread (1, 2 or 4), 0 = tuned default
                           (with `threads` given: the fewest that form a supported shape) */
    int schedule;       /* TPL_SCHED_* */
    int flags;          /* TPL_FLAG_* */
} tpl_opts;
/* Launch shapes (threads x residues per thread; a tile is their product):
 *  - backbone: threads 64, 128, 256, 512 x 1, 2, 4 (not 512 x 4); default 128 x 4;
 *  - full atom: 128, 256, 384 x 1; 128, 192 x 2; 64, 192 x 4; default 384 x 1.  A full-atom chain is cut into balanced tiles of at most
 *    threads x residues - 1 residues.  Rebuilding frames from the angles in
 *    the full-atom backward (TPL_BWD_RECOMPUTE, or TPL_BWD_AUTO without
 *    coordinates) needs one residue per thread: 128, 256 or 384 x 1 in both
 *    calls (TPL_ERR_INVALID_ARG otherwise). */

/* ------------------------------------------------------------------------ */
/* Backbone model (paper Section 3)                                          */
/* ------------------------------------------------------------------------ */

/* Bytes of workspace the backbone calls need for B chains of at most Lmax
 * residues.  The forward fills it (tile schedule, per-tile start frames); the
 * backward must get the same workspace, unmodified, with the same inputs and
 * options.  A backward given a workspace no forward filled sets
 * TPL_STATUS_BAD_WORKSPACE and writes zero gradients. */
size_t tpl_backbone_workspace_size(int B, int Lmax);

/* Section 3: r_i = R_0 R_1 ... R_i 0 with atom 3j = N (R(omega_j, pi-2.1186,
 * 1.330)), 3j+1 = CA (R(phi_j, pi-1.9391, 1.460)), 3j+2 = C (R(psi_j,
 * pi-2.0610, 1.525)); R(alpha, theta, d) is the Section 3 matrix.
 *   angles  [B][3][Lmax] in, lengths [B] int32 in (device),
 *   coords  [B][3*Lmax][3] out.
 * The chain is cut into tiles (threads x res_per_thread residues); persistent
 * CTAs take tiles from a work counter, scan the rigid transforms inside a tile
 * in parallel (FP32) and chain the tiles by a bounded look-back over the
 * earlier tiles' aggregates (re-orthonormalised). */
tpl_status tpl_backbone_forward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                float* coords, void* workspace, size_t workspace_bytes,
                                const tpl_opts* opts, tpl_stream stream);

/* Section 3, Eq. 2: grad_angles[b][r][j] = sum_i dL/dr_i . dr_i/dalpha, with
 * dr_i/dalpha = M_{k-1} dR_k/dalpha M_k^{-1} r_i, evaluated as
 * u_k . (sum_{i>=k} r_i x g_i - p_k x sum_{i>=k} g_i) by a reverse suffix scan
 * (u_k, p_k: axis and origin of frame k).
 *   grad_coords [B][3*Lmax][3] in, grad_angles [B][3][Lmax] out (0 at padding
 *   and at omega_0).  `coords` is the forward's output; it is read only in
 *   TPL_BWD_FROM_COORDS mode and may be NULL otherwise.  `workspace` is the
 *   one the forward filled. */
tpl_status tpl_backbone_backward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                 const float* coords, const float* grad_coords,
                                 float* grad_angles, void* workspace, size_t workspace_bytes,
                                 const tpl_opts* opts, tpl_stream stream);

/* ------------------------------------------------------------------------ */
/* Full-atom model (paper Section 2)                                         */
/* ------------------------------------------------------------------------ */

/* The backbone with the carbonyl O of every residue (the paper's backbone
 * model places N, CA and C only).  O_j is rigid in the frame of C_j after the
 * psi_j transform, where the full-atom tables put it (Section 2): bond C-O
 * 1.231 A, angle CA-C-O 120.1 degrees, dihedral N-CA-C-O = psi_j + 180, so
 * it lies in the plane of CA_j, C_j and N_{j+1}, opposite N_{j+1}; psi of the
 * last residue now moves an atom.  The scan places O with the residue's other
 * atoms (one more point per residue, 12 bytes written) and the backward
 * counts it among the atoms each angle moves (O_j after C_j: moved by every
 * angle up to psi_j).
 *   coords as tpl_backbone_forward; o_coords [B][Lmax][3] out (forward), in
 *   (backward with FROM_COORDS); grad_o [B][Lmax][3] in.
 *   Launch shapes 128 x 1, 2, 4 and 256 x 4 (default 128 x 4); workspace,
 *   schedule, bwd_mode and flags as tpl_backbone_forward / _backward (the
 *   backward with FROM_COORDS reads coords and o_coords; RECOMPUTE neither). */
tpl_status tpl_backbone_forward_o(const float* angles, const int32_t* lengths, int B, int Lmax, float* coords,
                                  float* o_coords, void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                  tpl_stream stream);
tpl_status tpl_backbone_backward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                   const float* coords, const float* o_coords, const float* grad_coords,
                                   const float* grad_o, float* grad_angles, void* workspace, size_t workspace_bytes,
                                   const tpl_opts* opts, tpl_stream stream);

/* The paper's own O(L^2) evaluation of Eq. 2 (Section 3): every (angle,
 * atom) term dL/dalpha_q = g_k . (M_{q-1} dR_q M_q^{-1} r_k), k >= q, summed
 * directly -- written as u_q . sum_{k >= q} (r_k - r_q) x g_k with u_q the unit
 * bond into atom q -- with no suffix scan: a comparator for
 * tpl_backbone_backward (same result to rounding, O(L^2) work per chain).
 *   coords: the backbone forward's output [B][3 Lmax][3]; grad_coords the
 *   same shape; grad_angles [B][3][Lmax] out (zeros at padding and for
 *   omega_0).  B <= 65535.  Needs no workspace. */
tpl_status tpl_backbone_backward_quadratic(const int32_t* lengths, int B, int Lmax, const float* coords,
                                           const float* grad_coords, float* grad_angles, tpl_stream stream);

/* The paper's depth-first evaluation of Eq. 1 (Section 2): for every angle,
 * the sum over the atoms it moves of g_k . (u x (r_k - p)) = u . ((r_k - p)
 * x g_k), u the unit axis and p a point on it, with no suffix scan -- O(L)
 * work per backbone angle, O(L^2) per chain: a comparator for
 * tpl_fullatom_backward (same result to rounding).  Angle j of a residue
 * moves the later residues and, in its own residue: phi all atoms but N,
 * psi C and O, omega all atoms, chi_k the side-chain groups k and beyond.
 *   seq, lengths, coords [B][Amax][3] (the full-atom forward's output),
 *   grad_coords the same shape; grad_angles [B][7][Lmax] out (zeros at
 *   padding, for omega_0 and for the chi angles a residue type lacks).
 *   B <= 65535.  Needs no workspace.  A chain with more atoms than Amax gets
 *   a zero gradient (the forward flags it). */
tpl_status tpl_fullatom_backward_quadratic(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                                           const float* coords, const float* grad_coords, float* grad_angles,
                                           tpl_stream stream);

/* Workspace of the full-atom calls; the same contract as the backbone's (the
 * backward reuses the forward's schedule and tile-start frames). */
size_t tpl_fullatom_workspace_size(int B, int Lmax);

/* Section 2: per residue M_1 = M_0 R_1(phi), side-chain frames M_1 R' R(chi_1)
 * R(chi_2) ..., M_3 = M_1 R_3(psi), next M_0 = M_3 R_4(omega_{j+1}); every atom
 * r = M_g r0 with r0 its standard-frame position in group g.
 *   angles [B][7][Lmax], seq [B][Lmax] uint8, lengths [B] int32 in;
 *   coords [B][Amax][3] out, num_atoms [B] int32 out. */
tpl_status tpl_fullatom_forward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                int B, int Lmax, int Amax, float* coords, int32_t* num_atoms,
                                void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                tpl_stream stream);

/* Section 2, Eq. 1: dL/dalpha_i = sum_{k in children(i)} g_k . (F_i r_k),
 * F_i = M_parent dR_i/dalpha M_i^{-1}, evaluated as u_i . (sum r_k x g_k -
 * p_i x sum g_k) with a suffix scan over residues for phi/psi/omega and a
 * suffix over the side-chain groups for chi.
 *   grad_coords [B][Amax][3] in, grad_angles [B][7][Lmax] out (0 at padding,
 *   unused chi rows and omega_0).  `workspace` is the one the forward filled,
 *   with the same options.  Axes and origins come from the forward's `coords`
 *   (TPL_BWD_FROM_COORDS, or TPL_BWD_AUTO with coords given), or frames are
 *   rebuilt from the angles and the forward's tile-start frames
 *   (TPL_BWD_RECOMPUTE, or AUTO with coords NULL: one residue per thread). */
tpl_status tpl_fullatom_backward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                 int B, int Lmax, int Amax, const float* coords,
                                 const float* grad_coords, float* grad_angles, void* workspace,
                                 size_t workspace_bytes, const tpl_opts* opts, tpl_stream stream);

/* Fused training step on the LRMSD loss of Section 4 chained into Eq. 1, in
 * two calls that share one workspace (the paper has no fused form; the
 * results equal tpl_fullatom_forward, tpl_lrmsd_forward with P = B and
 * Nmax = Amax, and tpl_fullatom_backward_lrmsd):
 *  - tpl_fullatom_lrmsd_forward: coords and num_atoms as tpl_fullatom_forward,
 *    lrmsd [B] = LRMSD(coords[b], target[b]) out: each tile also reduces its
 *    atoms' LRMSD moments against target [B][Amax][3]; then one CTA per chain
 *    sums its tiles' moments, solves for U and sums the squared residuals
 *    over the chain's atoms (FP64 final sum), leaving U, the centroids and
 *    1 / (N LRMSD) in the workspace (three kernel launches).
 *  - tpl_fullatom_lrmsd_backward: grad_angles = d(sum_b grad_lrmsd[b]
 *    LRMSD_b) / d(angles), each atom's LRMSD gradient formed inside the
 *    full-atom backward.  coords and target are those of the forward call.
 * Options as tpl_fullatom_forward; the schedule takes no packs here. */
size_t tpl_fullatom_lrmsd_workspace_size(int B, int Lmax);
tpl_status tpl_fullatom_lrmsd_forward(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                      int Lmax, int Amax, const float* target, float* coords, int32_t* num_atoms,
                                      float* lrmsd, void* workspace, size_t workspace_bytes, const tpl_opts* opts,
                                      tpl_stream stream);
tpl_status tpl_fullatom_lrmsd_backward(const uint8_t* seq, const int32_t* lengths, int B, int Lmax, int Amax,
                                       const float* coords, const float* target, const float* grad_lrmsd,
                                       float* grad_angles, void* workspace, size_t workspace_bytes,
                                       const tpl_opts* opts, tpl_stream stream);

/* Training step of the backbone model on the LRMSD loss (Section 3 forward,
 * Section 4 LRMSD, its gradient chained into Eq. 2, as the paper's training
 * does; the paper has no fused form), in one call:
 *   coords [B][3 Lmax][3] = the backbone forward (as tpl_backbone_forward);
 *   lrmsd [B] = LRMSD(coords[b], target[b]) over the 3 lengths[b] atoms;
 *   grad_angles [B][3][Lmax] = d(sum_b grad_lrmsd[b] LRMSD_b) / d(angles).
 * The results equal tpl_backbone_forward, tpl_lrmsd_forward (P = B, Nmax =
 * 3 Lmax, num_atoms = 3 lengths) and tpl_backbone_backward_lrmsd up to
 * rounding.  target [B][3 Lmax][3] and grad_lrmsd [B] are inputs; a chain
 * of at most one tile (threads x res_per_thread residues) is done by one CTA
 * with its coordinates and target in shared memory, so a batch with Lmax
 * at most one tile takes two kernel launches (work list, step).  Longer
 * chains add an eigen-solve launch and a backward launch.  workspace:
 * tpl_backbone_lrmsd_workspace_size(B, Lmax) bytes.  opts: launch shapes
 * 128 x 2, 128 x 4 (default), 256 x 2, 256 x 4, 512 x 2; bwd_mode RECOMPUTE
 * is rejected (the gradient is formed from the coordinates); the schedule
 * and TPL_FLAG_PADDING_ZEROED as for the chain calls.  A chain whose LRMSD
 * is 0 gets a zero gradient and sets TPL_STATUS_ZERO_LRMSD. */
size_t tpl_backbone_lrmsd_workspace_size(int B, int Lmax);
tpl_status tpl_backbone_lrmsd_step(const float* angles, const int32_t* lengths, int B, int Lmax,
                                   const float* target, const float* grad_lrmsd, float* coords, float* lrmsd,
                                   float* grad_angles, void* workspace, size_t workspace_bytes,
                                   const tpl_opts* opts, tpl_stream stream);

/* Backbone form of tpl_fullatom_backward_lrmsd below (Eq. 2 instead of
 * Eq. 1): grad_angles = d(sum_b grad_lrmsd[b] LRMSD(coords[b], target[b])) /
 * d(angles), equal to tpl_lrmsd_backward (P = B, Nmax = 3 Lmax, num_atoms =
 * 3 lengths) followed by tpl_backbone_backward with FROM_COORDS.
 *   coords: the backbone forward's output with `workspace`; target
 *   [B][3 Lmax][3]; lrmsd_workspace: as filled by tpl_lrmsd_forward on
 *   (coords, target, 3 lengths, P = B, Nmax = 3 Lmax).  The paper has no
 *   fused form. */
tpl_status tpl_backbone_backward_lrmsd(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* coords, const float* target, const float* grad_lrmsd,
                                       const void* lrmsd_workspace, size_t lrmsd_workspace_bytes,
                                       float* grad_angles, void* workspace, size_t workspace_bytes,
                                       const tpl_opts* opts, tpl_stream stream);

/* The backward of a training step on the LRMSD loss of Section 4 chained
 * into Eq. 1: grad_angles = d(sum_b grad_lrmsd[b] LRMSD(coords[b],
 * target[b])) / d(angles), the same as tpl_lrmsd_backward (P = B, Nmax =
 * Amax) followed by tpl_fullatom_backward with FROM_COORDS, with each atom's
 * coordinate gradient formed in the kernel from the coordinates, the target
 * and the per-pair state of the LRMSD forward, so no coordinate-gradient
 * tensor is written or read.  The paper has no fused form; it is this
 * library's fusion of two of its calls.
 *   coords: the full-atom forward's output with `workspace` (same inputs);
 *   target [B][Amax][3]; grad_lrmsd [B]; lrmsd_workspace: as filled by
 *   tpl_lrmsd_forward(coords, target, num_atoms of the forward, P = B,
 *   Nmax = Amax).  bwd_mode in opts is ignored. */
tpl_status tpl_fullatom_backward_lrmsd(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                       int B, int Lmax, int Amax, const float* coords, const float* target,
                                       const float* grad_lrmsd, const void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, const tpl_opts* opts, tpl_stream stream);

/* ------------------------------------------------------------------------ */
/* LRMSD (paper Section 4)                                                   */
/* ------------------------------------------------------------------------ */

/* Workspace for P pairs of at most Nmax atoms.  It carries the rotation U,
 * the centroids and LRMSD from the forward to the backward: pass the same
 * workspace, unmodified, to both. */
size_t tpl_lrmsd_workspace_size(int P, int Nmax);

/* Section 4: LRMSD(x = target, y = input) = min over rigid motions of
 * sqrt(sum |x_i - M y_i|^2 / N) by the quaternion method: centroids, R =
 * sum x' y'^T, the 4x4 matrix T(R), its largest eigenpair (lambda, q) from
 * an FP32 estimate (Newton on the characteristic polynomial and an adjugate
 * column, or cyclic Jacobi where lambda is nearly double) and one refinement
 * of q against the exact T (compensated double-float products and sums),
 * U(q); the value sum(|x'|^2 + |y'|^2) -
 * 2 lambda is evaluated in the equivalent residual form sum |y'_i - U x'_i|^2
 * (FP64 final reduction).
 *   input, target [P][Nmax][3], num_atoms [P] int32 in; lrmsd [P] float out. */
tpl_status tpl_lrmsd_forward(const float* input, const float* target, const int32_t* num_atoms,
                             int P, int Nmax, float* lrmsd, void* workspace,
                             size_t workspace_bytes, tpl_stream stream);

/* Kernels tpl_lrmsd_forward launches for P pairs on the current device: 1
 * for P > 0 (one CTA per pair does the moments, the eigen-solve and the
 * residuals; a wide CTA when the batch fits the GPU in one wave, a compact
 * one otherwise), 0 for P <= 0.  Needs no workspace; launches nothing. */
int tpl_lrmsd_forward_launches(int P);

/* Section 4: grad_input_i = grad_lrmsd[p] (y'_i - U x'_i) / (N LRMSD); 0 when
 * LRMSD < 1e-12 (status bit TPL_STATUS_ZERO_LRMSD).
 *   grad_lrmsd [P] in, grad_input [P][Nmax][3] out; `workspace` as filled by
 *   tpl_lrmsd_forward on the same inputs. */
tpl_status tpl_lrmsd_backward(const float* grad_lrmsd, const float* input, const float* target,
                              const int32_t* num_atoms, int P, int Nmax, float* grad_input,
                              const void* workspace, size_t workspace_bytes, tpl_stream stream);

/* Allocation-free variant of tpl_lrmsd_forward, for callers that can neither
 * allocate device memory nor pass a workspace (for example code whose device
 * memory is all owned by another runtime's allocator, or an interface without
 * a scratch argument).  The paper has no counterpart; this is an interface
 * convenience.  The scratch is a fixed array inside the library: every GPU
 * that loads the library holds it (256 KB) until the process exits.
 *   Limits: P <= 4096 pairs, Nmax <= 8192 atoms; larger sizes return
 *   TPL_ERR_BAD_SHAPE and launch nothing.  Inputs and outputs as in
 *   tpl_lrmsd_forward; no allocation, no workspace.
 *   The scratch used is the CURRENT device's: make the device that holds
 *   the pointers current before the call (the Python binding does).  The
 *   first call on a device looks up the scratch array's device address
 *   (once per device); make that first call before any stream capture.
 *   All calls share the one array and it keeps the last call's contents, so
 *   calls that overlap on the GPU (different streams without ordering between
 *   them) race; there is no backward companion (tpl_lrmsd_backward needs the
 *   workspace of tpl_lrmsd_forward). */
tpl_status tpl_lrmsd_forward_noalloc(const float* input, const float* target,
                                     const int32_t* num_atoms, int P, int Nmax, float* lrmsd,
                                     tpl_stream stream);

/* ------------------------------------------------------------------------ */
/* Plain FP64 per-chain forms: one CTA per chain (or pair), serial composition */
/* and serial suffix sums; the error reference and throughput comparator of   */
/* the FP32 scan kernels.  Same layouts with double; no workspace.            */
/* ------------------------------------------------------------------------ */

tpl_status tpl_backbone_forward_ref64(const double* angles, const int32_t* lengths, int B,
                                      int Lmax, double* coords, tpl_stream stream);
/* `coords` is this form's forward output (frames are read from it). */
tpl_status tpl_backbone_backward_ref64(const double* angles, const int32_t* lengths, int B,
                                       int Lmax, const double* coords, const double* grad_coords,
                                       double* grad_angles, tpl_stream stream);
tpl_status tpl_fullatom_forward_ref64(const double* angles, const uint8_t* seq,
                                      const int32_t* lengths, int B, int Lmax, int Amax,
                                      double* coords, int32_t* num_atoms, tpl_stream stream);
tpl_status tpl_fullatom_backward_ref64(const double* angles, const uint8_t* seq,
                                       const int32_t* lengths, int B, int Lmax, int Amax,
                                       const double* coords, const double* grad_coords,
                                       double* grad_angles, tpl_stream stream);
/* lrmsd_state [P][16] doubles (U row-major, centroids of x then y, LRMSD) is
 * written by the forward and read by the backward. */
tpl_status tpl_lrmsd_forward_ref64(const double* input, const double* target,
                                   const int32_t* num_atoms, int P, int Nmax, double* lrmsd,
                                   double* lrmsd_state, tpl_stream stream);
tpl_status tpl_lrmsd_backward_ref64(const double* grad_lrmsd, const double* input,
                                    const double* target, const int32_t* num_atoms, int P,
                                    int Nmax, const double* lrmsd_state, double* grad_input,
                                    tpl_stream stream);

/* ------------------------------------------------------------------------ */
/* Host helpers: residue tables, sizes, status                               */
/* ------------------------------------------------------------------------ */

/* Residue `code` (0..20): three-letter name (4 bytes with NUL), heavy-atom
 * count and number of free chi angles (Section 2: up to 7 angles per
 * residue).  Host only, no CUDA call. */
tpl_status tpl_residue_table(int code, char* three_letter, int* n_atoms, int* n_chi);

/* Atom `idx` of residue `code`: PDB name (8 bytes with NUL), rigid group
 * (0 = M_0 / N, 1 = M_1 / CA, 2 = M_3 / C and O, 3..6 = side-chain groups
 * 1..4) and its standard-frame position r0 (3 floats).  Host only. */
tpl_status tpl_residue_atom(int code, int idx, char* name, int* group, float* r0);

/* Atoms of chain b for a host sequence: sum of per-residue counts (-1 on a bad
 * code).  tpl_fullatom_max_atoms returns the maximum over the batch, i.e. the
 * smallest valid Amax before rounding up to a multiple of 4.  Host only. */
int tpl_fullatom_chain_atoms(const uint8_t* seq_host, int length);
int tpl_fullatom_max_atoms(const uint8_t* seq_host, const int32_t* lengths_host, int B, int Lmax);

/* Reads and clears the current device's status word (TPL_STATUS_* bits):
 * enqueues the read on `stream` and waits for that stream.  Not capturable. */
tpl_status tpl_get_status(tpl_stream stream, int* device_status);

/* Autotuner (the paper has no counterpart): runs forward + backward on the
 * caller's batch for every supported launch shape and schedule -- backbone:
 * threads 64..512 x residues per thread 1, 2, 4 x {PACKED, LONGEST_FIRST};
 * full atom: the seven shapes above (the one-residue ones for RECOMPUTE) x
 * {BATCH_ORDER, LONGEST_FIRST} -- times each as a CUDA graph of its calls
 * replayed between CUDA events on `stream` (one direct untimed pass, one
 * untimed replay, best of five), and writes the
 * fastest options to *best (and its time in ms to *best_ms if not NULL).
 * `bwd_mode` is kept in every candidate.  The arguments are those of the
 * forward and backward calls; coords, num_atoms and grad_angles are
 * overwritten.  It synchronizes `stream` and must not run while the stream is
 * being captured (TPL_ERR_INVALID_ARG).  Pass *best to later calls. */
tpl_status tpl_backbone_autotune(const float* angles, const int32_t* lengths, int B, int Lmax,
                                 float* coords, const float* grad_coords, float* grad_angles,
                                 void* workspace, size_t workspace_bytes, int bwd_mode, tpl_opts* best,
                                 float* best_ms, tpl_stream stream);
tpl_status tpl_fullatom_autotune(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                 int Lmax, int Amax, float* coords, int32_t* num_atoms,
                                 const float* grad_coords, float* grad_angles, void* workspace,
                                 size_t workspace_bytes, int bwd_mode, tpl_opts* best, float* best_ms,
                                 tpl_stream stream);

/* Autotuners of a training step on the LRMSD loss: as above, but each
 * candidate is timed on the three calls such a step makes -- the forward,
 * tpl_lrmsd_forward(coords, target, num_atoms, P = B, Nmax = 3 Lmax or Amax)
 * and the fused backward tpl_*_backward_lrmsd with grad_lrmsd [B] -- with
 * bwd_mode FROM_COORDS.  coords, lrmsd [B], lrmsd_workspace, grad_angles
 * (and num_atoms for the full atom) are overwritten; for the backbone,
 * num_atoms [B] = 3 lengths is an input. */
tpl_status tpl_backbone_lrmsd_autotune(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       float* coords, const float* target, const int32_t* num_atoms,
                                       const float* grad_lrmsd, float* lrmsd, void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, tpl_opts* best, float* best_ms, tpl_stream stream);
tpl_status tpl_fullatom_lrmsd_autotune(const float* angles, const uint8_t* seq, const int32_t* lengths, int B,
                                       int Lmax, int Amax, float* coords, int32_t* num_atoms, const float* target,
                                       const float* grad_lrmsd, float* lrmsd, void* lrmsd_workspace,
                                       size_t lrmsd_workspace_bytes, float* grad_angles, void* workspace,
                                       size_t workspace_bytes, tpl_opts* best, float* best_ms, tpl_stream stream);

/* Diagnostic (the paper has no counterpart): runs, in one thread of a
 * one-CTA launch on `stream`, the bounded wait that the chain kernels use
 * between CTAs, on the int at device address `flag`.  The caller keeps the
 * int at 0 (nothing sets it), so the wait gives up after its poll limit
 * (well under a second to a few seconds), sets TPL_STATUS_TIMEOUT and
 * returns; the context stays usable.  It shows that a lost cross-CTA signal
 * becomes a status bit, not a hang.  `flag` must be 4-byte aligned device
 * memory owned by the caller. */
tpl_status tpl_selftest_wait_timeout(const int* flag, tpl_stream stream);

/* Message of the last error returned on this thread ("" if none). */
const char* tpl_last_error(void);

/* Library version, "major.minor.patch". */
const char* tpl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TPL_H */
