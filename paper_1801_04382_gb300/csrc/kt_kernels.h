// Launchers of the CUDA kernels (internal interface between the host runtime and kt_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "kt_common.h"

// Lift a kernel's dynamic shared-memory limit to 227 KB on the current device.  The attribute is
// per device, so it is set once per (kernel, device) pair; only successes are remembered, a failed
// call is tried again on the next launch.
inline cudaError_t kt_allow_large_smem(const void *kern) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({kern, dev})) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess) done.insert({kern, dev});
  return e;
}

struct FwdArgs {
  int j;                 // interval 1..nt; 0 = prologue (update overlap at t_0 only)
  int nt;
  int update;            // propagate interval j with eps_old + deps (sequential Krotov update)
  int overlap;           // form the independent-trajectory overlap and Delta eps of interval j+1 here
  const int *pass_row;   // device: uniforms row of the running pass (written by init_pass)
  const void *psi_in;    // tile-layout states at t_{j-1}
  void *psi_out;         // tile-layout states at t_j
  const void *chi_t;     // tile-layout co-states at t_j (update only)
  const double *eps_old; // [n_ctrl][nt] pulse before this pass
  double *eps_new;       // [n_ctrl][nt] updated pulse (written by the last CTA)
  double *deps;          // [n_ctrl][nt] update
  const double *shape;   // [n_ctrl][nt]
  const double *U;       // [n_passes][M][draws]
  double *rstate;        // [M_pad] current threshold
  int *jcount;           // [M_pad] jumps so far in this pass
  int *rec_step;         // [M_pad][max_jumps]
  int *rec_ch;
  double *rec_s;
  double *rec_c;
  double *partials;      // [n_tiles][n_ctrl] (sharded: this shard's slice of the global array)
  unsigned *counter;     // last-CTA ticket, 0 between launches
  int finish;            // 1: the last CTA forms Delta eps from the partials; 0 (sharded): partials only
  KtCplx *tau;           // [M_pad] (j == nt)
  double *norm2;         // [M_pad] (j == nt)
  int *status;
  // whole forward sweep in one cooperative launch (one tile per CTA, every CTA resident): intervals
  // j .. nt, the state kept in shared memory between them; psi(t_i) goes to psi_ring[i & 1] (the
  // input of interval 1 is psi_in), chi(t_i) is read from chi_slots + i * slot_bytes.  With the
  // update the CTAs meet at a grid barrier (sync: two words, zero at the launch) after each
  // interval's overlap, and every CTA forms Delta eps from all tiles' partials in the finisher's
  // order (partials double-buffered by interval parity: [2][n_tiles][n_ctrl]).
  int sweep;
  void *psi_ring[2];
  const void *chi_slots;
  size_t slot_bytes;
  unsigned *sync;
};

struct BwdArgs {
  int j;                 // interval nt..1: chi(t_j) -> chi(t_{j-1})
  int nt;
  const void *chi_in;
  void *chi_out;
  const double *eps;     // [n_ctrl][nt] pulse of the recorded forward pass
  int *cursor;           // [M_pad] backward: latest unprocessed record; forward replay: next one
  int advance_cursor;
  int forward_replay;    // 1: psi(t_{j-1}) -> psi(t_j) under H_eff with the recorded jumps c L
  const int *jcount;     // [M_pad] records per trajectory (forward replay walks upwards)
  const int *rec_step;
  const int *rec_ch;
  const double *rec_s;
  const double *rec_c;
  int *status;
  // whole backward sweep in one launch (one tile per CTA): intervals j, j-1, ..., 1, the state kept
  // in shared memory between them; chi(t_{i-1}) of interval i goes to chi_slots + (i-1) * slot_bytes
  int sweep;
  void *chi_slots;
  size_t slot_bytes;
};

#include "../../include/krotov_traj.h"

// Record msg as the calling thread's last error (krotov_last_error) and return s.
kt_status kt_fail(kt_status s, const char *msg);

size_t kt_smem_bytes(const KtGeom &g, int elem_bytes, bool with_chi_buffer, bool with_next_buffer = false);
cudaError_t kt_launch_fwd(int fp64, int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops,
                          const FwdArgs &a, cudaStream_t st);
// Resident forward-kernel CTAs per SM for the launch shape of g (a whole-sweep launch needs every tile
// resident at once).
cudaError_t kt_fwd_blocks_per_sm(int fp64, int ept, const KtGeom &g, int *blocks);
cudaError_t kt_launch_bwd(int fp64, int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops,
                          const BwdArgs &a, cudaStream_t st);
cudaError_t kt_launch_fwd_f32(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a,
                              size_t smem, cudaStream_t st, int *occ = nullptr);
cudaError_t kt_launch_fwd_f64(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a,
                              size_t smem, cudaStream_t st, int *occ = nullptr);
cudaError_t kt_launch_bwd_f32(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const BwdArgs &a,
                              size_t smem, cudaStream_t st);
cudaError_t kt_launch_bwd_f64(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const BwdArgs &a,
                              size_t smem, cudaStream_t st);
// pass[0] = uniforms row of the next pass, pass[1] = rows held, pass[2] = row of the running pass.
// init_pass takes pass[0] for the new pass, advances it cyclically and resets thresholds and counts.
cudaError_t kt_launch_init_pass(const KtGeom &g, const double *U, int *pass, double *rstate, int *jcount,
                                cudaStream_t st);
// pass[0] = 0, pass[1] = n_passes
cudaError_t kt_launch_pass_reset(int *pass, int n_passes, cudaStream_t st);
// nu[c] = noise of pulse c minus ref (nullable) (five-point cubic Savitzky-Golay residual, integrated), nt >= 5
cudaError_t kt_launch_pulse_noise(const double *eps, const double *ref, int n_ctrl, int nt, double dt, double *nu,
                                  cudaStream_t st);
cudaError_t kt_launch_cursor_seek(const KtGeom &g, const int *rec_step, const int *jcount, int upto,
                                  int *cursor, cudaStream_t st);
// cursor[k] = first record of trajectory k with interval >= from (jcount[k] if none)
cudaError_t kt_launch_cursor_seek_fwd(const KtGeom &g, const int *rec_step, const int *jcount, int from,
                                      int *cursor, cudaStream_t st);
// Cross-trajectory update of interval j+1 (Eq. cross_traj_update) from psi(t_j), xi(t_j) in tile
// layout: transposes both to [x][k] (k padded to a multiple of 32), applies the control factors,
// sums Im[<xi_k|h_c|psi_k'><psi_k'|xi_k>] over all pairs in 32 x 32 pair tiles and, in the last
// CTA, writes deps / eps_new of interval j+1 (0-based index j).
struct CrossArgs {
  int j, nt;
  const void *psi;       // tile layout, t_j
  const void *xi;        // tile layout, t_j
  void *X, *P, *HP;      // [d][Mp], [d][Mp], [n_ctrl][d][Mp] work arrays
  double *pairbuf;       // [slices][Mp][Mp][1 + n_ctrl] FP64 complex slice sums of G and A_c
  double *partials;      // [(Mp/32)^2][n_ctrl]
  unsigned *counter;
  const double *eps_old;
  double *eps_new, *deps;
  const double *shape;
  int *status;
};
size_t kt_cross_work_bytes(const KtGeom &g, int elem_bytes);   // X + P + HP
size_t kt_cross_partials(const KtGeom &g);                     // entries of CrossArgs::partials
int kt_cross_slices(const KtGeom &g);                          // slices of the element range
size_t kt_cross_pair_bytes(const KtGeom &g);                   // CrossArgs::pairbuf
cudaError_t kt_launch_cross(int fp64, const KtGeom &g, const KtOps &ops, const CrossArgs &a, cudaStream_t st);

cudaError_t kt_launch_chi_grad_boundary(int fp64, const KtGeom &g, const KtOps &ops, const KtCplx *tau,
                                        const double *norm2, const void *psi, void *chi, cudaStream_t st);

// Gradient of the frozen-record trajectory functional on interval j (one CTA per trajectory).
struct GradArgs {
  int j, nt;
  const void *psi_prev;  // tile-layout psi(t_{j-1}) of the recorded forward pass
  const void *chi_t;     // tile-layout chi~(t_j)
  const double *eps;     // [n_ctrl][nt]
  const int *cursor;     // [M_pad] latest record with interval <= j (backward cursor, not advanced)
  const int *rec_step;
  const int *rec_ch;
  const double *rec_s;
  const double *rec_c;
  double *partials;      // [M][n_ctrl]
  unsigned *counter;
  double *grad;          // [n_ctrl][nt]: dJ_T/deps of interval j written by the last CTA
  int *status;
};
// g1: the problem geometry re-cut to one trajectory per CTA (T = 1)
size_t kt_grad_smem_bytes(const KtGeom &g1, int elem_bytes);
cudaError_t kt_launch_grad(int fp64, int ept, const KtGeom &g1, int T_layout, int tile_elems_layout,
                           const KtGenImage &im_fwd, const KtGenImage &im_bwd, const KtOps &ops, const GradArgs &a,
                           cudaStream_t st);

// Delta eps and the new pulse of interval j+1 (0-based index j) from the tile partials of all shards
// [n_tiles][n_ctrl]: one block of g.nthreads threads summing in the order of the forward kernel's
// last-CTA finisher (thread chunks of tiles, shuffle tree, warps in order), so a sharded problem
// gives the single-GPU result bit for bit.
cudaError_t kt_launch_finish_update(const KtGeom &g, int n_tiles, const double *partials, int j, int nt,
                                    const double *shape, const double *eps_old, double *deps, double *eps_new,
                                    int *status, cudaStream_t st);
// status <- KT_DEV_NONFINITE / KT_DEV_RANGE if a value of eps [n] is not finite or |eps| > bound
cudaError_t kt_launch_pulse_check(const double *eps, long long n, double bound, int *status, cudaStream_t st);
// JT[0] = 1 - (1/M) sum_k |tau_k|^2, or 1 - Re tau_0 for a density matrix
cudaError_t kt_launch_functional(const KtCplx *tau, int M, int density, double *JT, cudaStream_t st);

cudaError_t kt_launch_chi_boundary(int fp64, const KtGeom &g, const KtOps &ops, const KtCplx *tau, void *chi,
                                   cudaStream_t st);
