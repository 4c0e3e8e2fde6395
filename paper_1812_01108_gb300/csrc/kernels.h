// Host-side launchers of the sm_103a kernels (called by the C ABI in api.cu).
// Every launcher enqueues on `stream`, returns the launch error (cudaSuccess
// when all launches were accepted) and never synchronises.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tpl.h"  // TPL_FLAG_*

namespace tpl {

struct LaunchCfg {
    int threads;        // CTA size
    int res_per_thread; // consecutive residues per thread (tile = threads * res_per_thread)
    int flags = 0;      // TPL_FLAG_*
    bool packed = false;  // full atom: the work list may hold packs of whole chains
};

// Bytes of the chain workspace (tile list, look-back flags and aggregates,
// tile-start frames; with per_residue, each residue's first atom; with step,
// the fused training step's per-tile LRMSD partials) for B chains of at most
// Lmax residues.
size_t chain_ws_bytes(int B, int Lmax, bool per_residue, bool step);

// CTAs of a persistent launch of `kernel`: SMs x resident CTAs per SM (cached
// per kernel and device).
int persistent_grid(const void* kernel, int threads, size_t smem);

// K1 / K2: backbone FP32 scan kernels.
bool backbone_cfg_supported(int threads, int res_per_thread);
cudaError_t launch_backbone_forward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                    float* coords, int sched_mode, void* workspace,
                                    LaunchCfg cfg, cudaStream_t s);
// K2q: the paper's O(L^2) form of Eq. 2 from the forward's coordinates (comparator).
cudaError_t launch_backbone_backward_quadratic(const int32_t* lengths, int B, int Lmax, const float* coords,
                                              const float* grad_coords, float* grad_angles, cudaStream_t s);
cudaError_t launch_backbone_backward(const float* angles, const int32_t* lengths, int B, int Lmax,
                                     const float* coords, const float* grad_coords,
                                     float* grad_angles, bool from_coords, void* workspace,
                                     LaunchCfg cfg, cudaStream_t s);

// K1 / K2 with the carbonyl O of every residue: o_coords [B][Lmax][3] out of
// the forward; the backward adds grad_o on those atoms (o_coords read with
// from_coords).
bool backbone_o_cfg_supported(int threads, int res_per_thread);
cudaError_t launch_backbone_forward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                      float* coords, float* o_coords, int sched_mode, void* workspace,
                                      LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_backbone_backward_o(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* coords, const float* o_coords, const float* grad_coords,
                                       const float* grad_o, float* grad_angles, bool from_coords,
                                       void* workspace, LaunchCfg cfg, cudaStream_t s);

// K2 with the LRMSD gradient formed in place of a coordinate-gradient input
// (P = B pairs of Nmax = 3 Lmax atoms).
cudaError_t launch_backbone_backward_lrmsd(const float* angles, const int32_t* lengths, int B, int Lmax,
                                           const float* coords, const float* target,
                                           const float* grad_lrmsd, const float* lrmsd_state,
                                           float* grad_angles, void* workspace, LaunchCfg cfg,
                                           cudaStream_t s);

// K3 / K4: full-atom FP32 scan kernels.
bool fullatom_cfg_supported(int threads, int res_per_thread);
cudaError_t launch_fullatom_forward(const float* angles, const uint8_t* seq,
                                    const int32_t* lengths, int B, int Lmax, int Amax,
                                    float* coords, int32_t* num_atoms, int sched_mode,
                                    void* workspace, LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_fullatom_backward(const float* angles, const uint8_t* seq,
                                     const int32_t* lengths, int B, int Lmax, int Amax,
                                     const float* coords, const float* grad_coords,
                                     float* grad_angles, bool from_coords, void* workspace,
                                     LaunchCfg cfg, cudaStream_t s);

// K4q: the paper's depth-first O(L^2) form of Eq. 1 from the forward's
// coordinates (comparator).
cudaError_t launch_fullatom_backward_quadratic(const uint8_t* seq, const int32_t* lengths, int B, int Lmax,
                                              int Amax, const float* coords, const float* grad_coords,
                                              float* grad_angles, cudaStream_t s);

// K4 with the LRMSD gradient formed in place of a coordinate-gradient input:
// the gradient of sum_b grad_lrmsd[b] LRMSD(coords[b], target[b]).
cudaError_t launch_fullatom_backward_lrmsd(const uint8_t* seq, const int32_t* lengths, int B, int Lmax,
                                          int Amax, const float* coords, const float* target,
                                          const float* grad_lrmsd, const float* lrmsd_state,
                                          float* grad_angles, void* workspace, LaunchCfg cfg,
                                          cudaStream_t s);

// The eigen-solve of K5 on per-tile moment partials (slot = chain * tiles_max
// + tile, 20 floats each; chain p cut into balanced full-atom tiles or into
// tiles of `tile` residues): the fused training steps.  Writes the per-pair
// state (16 floats per pair) of the chains of at least min_tiles tiles.
// num_atoms null: chain p has 3 lengths[p] atoms (backbone).
// Fused full-atom step: per chain, its tile moments summed, the eigen-solve, the
// residual pass over its atoms; state (as tpl_lrmsd_forward's) and lrmsd out.
cudaError_t launch_lrmsd_parts(const float* input, const float* target, const int32_t* num_atoms, int P,
                               int Nmax, const float* tile_moments, int tiles_max, const int32_t* lengths, int tile,
                               int Lmax, float* state, float* lrmsd, cudaStream_t s);
cudaError_t launch_lrmsd_solve_tiles(const float* input, const float* target, const int32_t* num_atoms,
                                     int P, int Nmax, const float* tile_moments, int tiles_max,
                                     const int32_t* lengths, int tile, int Lmax, float* state,
                                     cudaStream_t s, bool balanced, int min_tiles);

// Training step of the backbone model on the LRMSD loss (K1s, workspace of
// chain_ws_bytes(B, Lmax, false, true)): coordinates, LRMSD per chain and the
// gradient of sum_b grad_lrmsd[b] LRMSD_b.
bool backbone_step_cfg_supported(int threads, int res_per_thread);
cudaError_t launch_backbone_lrmsd_step(const float* angles, const int32_t* lengths, int B, int Lmax,
                                       const float* target, const float* grad_lrmsd, float* coords,
                                       float* lrmsd, float* grad_angles, int sched_mode, void* workspace,
                                       LaunchCfg cfg, cudaStream_t s);

// Fused training step on the full-atom model with the LRMSD loss (workspace of
// chain_ws_bytes(B, Lmax, true, true)): forward = schedule, forward with
// per-tile LRMSD moments, per chain the eigen-solve and the residual pass
// (LRMSD out); backward = the full-atom backward with the LRMSD gradient
// formed inside.
cudaError_t launch_fullatom_lrmsd_forward(const float* angles, const uint8_t* seq, const int32_t* lengths,
                                          const float* target, int B, int Lmax, int Amax, float* coords,
                                          int32_t* num_atoms, float* lrmsd, int sched_mode, void* workspace,
                                          LaunchCfg cfg, cudaStream_t s);
cudaError_t launch_fullatom_lrmsd_backward(const uint8_t* seq, const int32_t* lengths, const float* coords,
                                           const float* target, const float* grad_lrmsd, int B, int Lmax,
                                           int Amax, float* grad_angles, void* workspace, LaunchCfg cfg,
                                           cudaStream_t s);

// K5 / K6: LRMSD.  The workspace layout is private to lrmsd.cu.
size_t lrmsd_ws_bytes(int P, int Nmax);
// Per-pair state the LRMSD forward leaves in its workspace: U (9, row-major),
// centroid of the target, centroid of the input, 1 / (N LRMSD) (16 floats).
const float* lrmsd_state(const void* ws, int P, int Nmax);
// Kernels tpl_lrmsd_forward launches for P pairs on the current device.
int lrmsd_forward_launches(int P);
cudaError_t launch_lrmsd_forward(const float* input, const float* target,
                                 const int32_t* num_atoms, int P, int Nmax, float* lrmsd,
                                 void* ws, cudaStream_t s);
cudaError_t launch_lrmsd_backward(const float* grad_lrmsd, const float* input,
                                  const float* target, const int32_t* num_atoms, int P, int Nmax,
                                  float* grad_input, const void* ws, cudaStream_t s);

// LRMSD forward with its scratch in a fixed device array (no workspace, no
// allocation); sizes above the maxima are rejected by the caller.
int lrmsd_noalloc_max_pairs();
int lrmsd_noalloc_max_atoms();
size_t lrmsd_noalloc_scratch_bytes();
cudaError_t launch_lrmsd_forward_noalloc(const float* input, const float* target,
                                         const int32_t* num_atoms, int P, int Nmax, float* lrmsd,
                                         cudaStream_t s);

// K7: plain FP64 per-chain forms.
cudaError_t launch_backbone_forward_ref64(const double* angles, const int32_t* lengths, int B,
                                          int Lmax, double* coords, cudaStream_t s);
cudaError_t launch_backbone_backward_ref64(const double* angles, const int32_t* lengths, int B,
                                           int Lmax, const double* coords,
                                           const double* grad_coords, double* grad_angles,
                                           cudaStream_t s);
cudaError_t launch_fullatom_forward_ref64(const double* angles, const uint8_t* seq,
                                          const int32_t* lengths, int B, int Lmax, int Amax,
                                          double* coords, int32_t* num_atoms, cudaStream_t s);
cudaError_t launch_fullatom_backward_ref64(const double* angles, const uint8_t* seq,
                                           const int32_t* lengths, int B, int Lmax, int Amax,
                                           const double* coords, const double* grad_coords,
                                           double* grad_angles, cudaStream_t s);
cudaError_t launch_lrmsd_forward_ref64(const double* input, const double* target,
                                       const int32_t* num_atoms, int P, int Nmax, double* lrmsd,
                                       double* state, cudaStream_t s);
cudaError_t launch_lrmsd_backward_ref64(const double* grad_lrmsd, const double* input,
                                        const double* target, const int32_t* num_atoms, int P,
                                        int Nmax, const double* state, double* grad_input,
                                        cudaStream_t s);

// Reads and clears the device status word (blocking on `s`).
cudaError_t read_and_clear_status(cudaStream_t s, int* out);

}  // namespace tpl
