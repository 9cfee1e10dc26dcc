// Internal definitions shared by the host runtime and the CUDA kernels.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define KT_HD __host__ __device__ __forceinline__
#else
#define KT_HD inline
#endif

#define KT_MAX_NODES 8
#define KT_MAX_CTRL 8
#define KT_MAX_CTERMS 16  // control terms (a control acting on one node; two per control in Liouville space)
#define KT_MAX_LIND 4
#define KT_MAX_PAIRS 28
#define KT_MAX_NL 9       // local dimension of the cavity-structure kernels (atom x cavity, cutoff <= 2)
#define KT_MAX_S 4        // off-diagonal entries per row of a node-local generator factor
#define KT_MAX_SH 6       // entries per row of a control factor (update overlap)
#define KT_MAX_K 96       // Chebyshev terms
#define KT_MAX_T 32       // trajectories per tile
#define KT_MAX_ROUNDS 16  // jump-separated pieces of one interval in one kernel

// Kernel families timed by krotov_set_profiling (mirror KT_PROF_* in the public header).
#ifndef KT_PROF_FAMILIES
#define KT_PROF_FAMILIES 5
#define KT_PROF_FWD 0
#define KT_PROF_BWD 1
#define KT_PROF_GRAD 2
#define KT_PROF_CROSS 3
#define KT_PROF_FINISH 4
#endif

// Device status word values (first error wins); mirror kt_status.
#define KT_DEV_OK 0
#define KT_DEV_NONFINITE 5
#define KT_DEV_RECORD_FULL 6
#define KT_DEV_RANGE 8
#define KT_DEV_ZERO_JUMP 9
#define KT_DEV_TIMEOUT 4

// Chebyshev expansion of exp(-i G s) with G = c + r * Ghat (Ghat's spectrum in an ellipse
// around [-1, 1]):  exp(-i G s) = exp(-i c s) sum_k (2 - delta_k0) (-i)^k J_k(r s) T_k(Ghat).
//
// Bessel functions J_0..J_{n-1}(alpha) by Miller's backward recurrence
//   J_{k-1} = (2k / alpha) J_k - J_{k+1},
// started far above the wanted orders from (0, tiny) and normalised with the Neumann
// identity J_0 + 2 sum_{m >= 1} J_{2m} = 1 (J.C.P. Miller, 1952; Numerical Recipes' bessj).
// Values are rescaled whenever they grow past 1e150 so that tiny alpha cannot overflow.
KT_HD int kt_bessel_miller(double alpha, int n, double *out) {
  if (n < 1 || n > 256 || !(alpha >= 0.0)) return -1;
  if (alpha < 1e-290) {
    out[0] = 1.0;
    for (int k = 1; k < n; ++k) out[k] = 0.0;
    return 0;
  }
  int start = n + 20 + (int)(alpha);
  start += (start & 1);                 // even start keeps the Neumann sum bookkeeping simple
  for (int k = 0; k < n; ++k) out[k] = 0.0;
  double jp1 = 0.0, jk = 1e-200, norm = 0.0;
  const double inv = 2.0 / alpha;
  for (int k = start; k >= 1; --k) {
    double jm1 = (double)k * inv * jk - jp1;
    jp1 = jk;
    jk = jm1;                            // jk now holds J_{k-1}
    int km1 = k - 1;
    if (km1 < n) out[km1] = jk;
    if (km1 > 0 && (km1 & 1) == 0) norm += 2.0 * jk;
    if (jk > 1e150 || jk < -1e150) {
      jk *= 1e-150; jp1 *= 1e-150; norm *= 1e-150;
      for (int q = km1; q < n; ++q) out[q] *= 1e-150;
    }
  }
  norm += jk;                            // + J_0
  const double s = 1.0 / norm;
  for (int k = 0; k < n; ++k) out[k] *= s;
  return 0;
}

struct KtCplx { double re, im; };

// Problem geometry and constants passed to every kernel by value.
struct KtGeom {
  int n_nodes, n_loc, d, T;          // T = trajectories per tile (interleaved, element-major)
  int tile_elems;                    // complex elements per tile in global memory (>= d*T, multiple of 4)
  int n_tiles, M, M_pad, nthreads;
  int S, SH, n_pairs, n_ctrl, n_lind;
  int K;                             // Chebyshev terms of a full step
  int max_jumps, draws;              // jump cap and uniforms per trajectory and pass
  int prefetch_chi;                  // forward kernel keeps a third tile buffer for chi(t_j)
  int bwd_grid;                      // > 0: backward kernel CTAs looping over tiles, next input prefetched
  int fwd_grid;                      // > 0: the same for the forward kernel (psi and chi of the next tile prefetched)
  int first_order;                   // jump scheme: 0 jump times by bisection, 1 at most one jump per interval, at its end
  int stride[KT_MAX_NODES];          // element stride of node i (n_loc^(N-1-i))
  int ctrl_node[KT_MAX_CTRL];        // node of control c (its ket node for a density matrix)
  int n_cterms;                      // control terms: control cterm_ctrl[t] acting on node cterm_node[t]
  int cterm_ctrl[KT_MAX_CTERMS];
  int cterm_node[KT_MAX_CTERMS];
  int density;                       // 1: the one "trajectory" is vec(rho) in Liouville space (no jumps, no normalisation)
  double M_norm;                     // M of the update's 1/M: all trajectories of the problem (M, or M_total when sharded)
  int inject_timeout;                // test of the failure path: the first wait for a bulk copy runs out
  double lam[KT_MAX_CTRL];
  double dt, eps_bound;
  double c_fwd, c_bwd, r;            // generator centre (per direction) and half width
};

// Precomputed (pulse independent) generator tables of one direction, FP64, in global memory.
struct KtGenImage {
  const int *loc_dl;          // [N][n_loc][S] local column delta y - x (0 = no entry)
  const KtCplx *loc_base;     // [N][n_loc][S] scaled (1/r) drift part
  const KtCplx *ctrl_slot;    // [n_cterms][n_loc][S] scaled per-unit-eps part of term t on node cterm_node[t]
  const KtCplx *diag_base;    // [N][n_loc] scaled diagonal (node 0 also holds -c/r)
  const KtCplx *ctrl_diag;    // [n_cterms][n_loc] scaled per-unit-eps diagonal part
  const int *pair_off;        // [P][n_loc*n_loc] element offset (in elements, before *T); 0 = none
  const KtCplx *pair_val;     // [P][n_loc*n_loc] scaled
  const KtCplx *cheb_full;    // [K] full-step coefficients, phase exp(-i c dt) folded in
  const KtCplx *pair_coef;    // [P] scaled coefficient of pair term p (value = coef * a^dag a entries)
  int pair_dst[KT_MAX_PAIRS]; // node raised by pair term p of this direction
  int pair_src[KT_MAX_PAIRS]; // node lowered by pair term p of this direction
  // Cavity-structure kernels with real / imaginary coupling classes: the pulse-independent
  // coefficients that every Chebyshev term reads, as kernel-parameter constants in both precisions
  // (the kernels then take them as constant-bank operands instead of shared-memory loads).
  float kd32[2 * KT_MAX_NL];  // last node's diagonal, (re, im) per local index
  double kd64[2 * KT_MAX_NL];
  float kc32[2 * 2];          // last node's cavity couplings: [n-1] row (r, n-1) <- (g, n), [NC + n-1] the reverse
  double kc64[2 * 2];
  float kp32[KT_MAX_PAIRS];   // imaginary part of pair coefficient p
  double kp64[KT_MAX_PAIRS];
};

// Pulse-independent operators shared by both directions.
struct KtOps {
  const int *lo_dl;           // [n_loc] ladder factor a: row x -> column x + lo_dl[x]
  const KtCplx *lo_val;       // [n_loc] value (0 = empty row)
  const int *ra_dl;           // [n_loc] adjoint a^dag: row x -> column x + ra_dl[x]
  const KtCplx *ra_val;       // [n_loc]
  const KtCplx *lind_coef;    // [n_lind][N]
  const int *hc_dl;           // [n_cterms][n_loc][SH] control term factor (unscaled), column delta
  const KtCplx *hc_val;       // [n_cterms][n_loc][SH] (0 = no entry)
  const uint32_t *digits;     // [d] node digits of each basis index, node i in bits 4i..4i+3
  const KtCplx *tgt;          // [d] target state
};
