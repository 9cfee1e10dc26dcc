#pragma once
// CUDA kernels of the trajectory-parallel Krotov hot path (sm_103a).
//
// One CTA owns a tile of T trajectories for one time interval.  The tile's states sit in
// global memory as [d][T] complex (element-major, trajectories interleaved), so that a warp
// whose items share an element index (T = 32) runs the structured generator uniformly and
// reads its neighbours from consecutive shared-memory words.
//
// Per interval the CTA applies exp(-i G dt) by a Chebyshev series (paper Sec. 2.1: exact
// propagation over long steps, the basic operation being the matrix-vector product of
// Sec. 2.3), keeping T_{k-1}/T_{k+1} and T_k in two shared-memory buffers and the running
// sum in registers.  G is never formed: it is the sum of node-local factors, pair hops
// a_dst^dag a_src and a diagonal, all read from small per-interval tables in shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kt_common.h"
#include "kt_kernels.h"

namespace kt {

template <typename R> struct C2;
template <> struct C2<float> { typedef float2 T; };
template <> struct C2<double> { typedef double2 T; };

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cfma(C a, C b, C c) {  // c + a*b
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}

// c + a*b for a purely real (rfma, a) or purely imaginary (ifma, i b) coefficient: the two
// FMAs of cfma whose coefficient part is nonzero, in cfma's order, so the result is bit-identical.
template <typename C, typename R> __device__ __forceinline__ C rfma(R a, C b, C c) {
  c.x = fma(a, b.x, c.x);
  c.y = fma(a, b.y, c.y);
  return c;
}
template <typename C, typename R> __device__ __forceinline__ C ifma(R bi, C b, C c) {
  c.x = fma(-bi, b.y, c.x);
  c.y = fma(bi, b.x, c.y);
  return c;
}

template <typename C> __device__ __forceinline__ C from_kc(KtCplx z) {
  typedef decltype(C().x) R;
  return mkc((R)z.re, (R)z.im);
}

__device__ __forceinline__ void set_status(int *status, int code) {
  atomicCAS(status, KT_DEV_OK, code);
}

// ---- bulk (TMA) copies between global and shared memory, completing on an mbarrier -------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// one thread: arm the barrier for `bytes` and start the copy global -> shared
// (addresses 16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                          unsigned long long *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

#define KT_WAIT_CYCLES 4000000000LL   // ~2 s of SM clock

// wait (one thread) for phase `phase` of the barrier, giving up after `budget` cycles of clock
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t phase,
                                                  long long budget = KT_WAIT_CYCLES) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > budget) return false;
  return true;
}

// one thread: copy shared -> global (16-byte aligned, size a multiple of 16) as one bulk group
__device__ __forceinline__ void bulk_store(void *dst_gmem, const void *src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem), "r"(smem_u32(src_smem)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_store_wait() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier of all CTAs of a cooperative launch (every CTA resident by the launch's guarantee):
// sync[0] counts arrivals, the last arrival resets it and moves the generation sync[1] on to `gen`
// + 1 (both words zero at the launch, gen counting the barriers passed).  Every write a CTA made
// before the barrier is visible to every CTA after it.  Bounded: a CTA that waits longer than
// KT_WAIT_CYCLES records KT_DEV_TIMEOUT and sees false (the launch's results are then void).
__device__ __forceinline__ bool grid_barrier(unsigned *sync, unsigned gen, int *flag_slot, int *status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    __threadfence();
    if (atomicAdd(&sync[0], 1u) == gridDim.x - 1) {
      atomicExch(&sync[0], 0u);
      __threadfence();
      atomicExch(&sync[1], gen + 1);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu(&sync[1]) != gen + 1) {
        if (clock64() - t0 > KT_WAIT_CYCLES) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!ok) set_status(status, KT_DEV_TIMEOUT);
    *flag_slot = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag_slot != 0;
}

// Whole-tile load by the bulk engine: thread 0 waits (bounded, ~2 s) and the block learns the
// outcome.  On a timeout the status word gets KT_DEV_TIMEOUT, thread 0 waits once more (~2 s) so
// that the copy in flight lands before the block leaves, and false is returned to every thread.
// idle_bar (a test of this failure path, kt_config.inject_copy_timeout): the first wait watches a
// barrier nothing arrives at, for ~10 us, so that the timeout path runs deterministically.
__device__ __forceinline__ bool tile_wait(unsigned long long *bar, uint32_t phase, int *flag_slot, int *status,
                                          unsigned long long *idle_bar) {
  if (threadIdx.x == 0) {
    const bool ok = idle_bar ? mbar_wait_bounded(idle_bar, 0, 20000) : mbar_wait_bounded(bar, phase);
    if (!ok) {
      set_status(status, KT_DEV_TIMEOUT);
      mbar_wait_bounded(bar, phase);   // give the copy in flight a second bounded chance to land
    }
    *flag_slot = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag_slot != 0;
}

// --------------------------------------------------------------------------------------
// Shared-memory carve-up (identical on host and device; see kt_smem_bytes).
struct Smem {
  void *bufA, *bufB;          // [tile_elems] complex each
  void *bufC;                 // [tile_elems] prefetched chi(t_j) (forward kernel, when it fits)
  void *bufD;                 // [tile_elems] the next tile's prefetched psi (forward kernel looping over tiles)
  unsigned long long *mbar;   // [4] transaction barriers of the bulk copies ([0], [3] psi, [1] chi); [2] never receives an arrival
  int *loc_off;               // [N*n_loc*S]  element offset * T (0 = no entry)
  void *loc_val;              // [N*n_loc*S]
  void *diag;                 // [N*n_loc]
  int *pair_off;              // [P*n_loc^2]
  void *pair_val;             // [P*n_loc^2]
  int *hc_off;                // [n_cterms*n_loc*SH]
  void *hc_val;               // [n_cterms*n_loc*SH]
  void *coef;                 // [K][T]
  double *red;                // [nwarps][T][8]
  double *tsc;                // per-trajectory scalars [16][T]
  int *tin;                   // per-trajectory ints [16][T]
  double *eps;                // [n_ctrl]
  int *flag;                  // [8] block flags
  void *ldense;               // [n_loc][n_loc] last node's factor, dense (cavity-structure path)
  void *lora;                 // [2][n_loc] ladder values a (row x) and a^dag (row x)
  void *pcoef;                // [P] scaled pair coefficients
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline size_t carve(const KtGeom &g, int esz, char *base, Smem *s, bool with_c,
                                        bool with_d = false) {
  const int nl2 = g.n_loc * g.n_loc;
  const int nwarps = g.nthreads / 32;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char * {
    off = align_up(off, 16);
    char *p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const size_t tile = (size_t)g.tile_elems * esz;
  char *a = take(tile), *b = take(tile);
  char *cbuf = with_c ? take(tile) : nullptr;
  char *dbuf = with_d ? take(tile) : nullptr;
  char *mb = take(4 * sizeof(unsigned long long));
  char *lo = take(sizeof(int) * g.n_nodes * g.n_loc * g.S);
  char *lv = take((size_t)esz * g.n_nodes * g.n_loc * g.S);
  char *dg = take((size_t)esz * g.n_nodes * g.n_loc);
  char *po = take(sizeof(int) * g.n_pairs * nl2);
  char *pv = take((size_t)esz * g.n_pairs * nl2);
  char *ho = take(sizeof(int) * g.n_cterms * g.n_loc * g.SH);
  char *hv = take((size_t)esz * g.n_cterms * g.n_loc * g.SH);
  char *cf = take((size_t)esz * g.K * g.T);
  char *rd = take(sizeof(double) * nwarps * g.T * 8);
  char *ts = take(sizeof(double) * 16 * g.T);
  char *ti = take(sizeof(int) * 16 * g.T);
  char *ep = take(sizeof(double) * KT_MAX_CTRL);
  char *fl = take(sizeof(int) * 8);
  char *ld = take((size_t)esz * g.n_loc * g.n_loc);
  char *lr = take((size_t)esz * 2 * g.n_loc);
  char *pc = take((size_t)esz * (g.n_pairs > 0 ? g.n_pairs : 1));
  if (s) {
    s->bufA = a; s->bufB = b; s->bufC = cbuf; s->bufD = dbuf; s->mbar = (unsigned long long *)mb; s->loc_off = (int *)lo; s->loc_val = lv; s->diag = dg;
    s->pair_off = (int *)po; s->pair_val = pv; s->hc_off = (int *)ho; s->hc_val = hv;
    s->coef = cf; s->red = (double *)rd; s->tsc = (double *)ts; s->tin = (int *)ti;
    s->eps = (double *)ep; s->flag = (int *)fl;
    s->ldense = ld; s->lora = lr; s->pcoef = pc;
  }
  return align_up(off, 16);
}

// per-trajectory scalar slots in Smem::tsc / Smem::tin
enum { TS_R = 0, TS_LO, TS_HI, TS_S0, TS_LEN, TS_NRM, TS_C, TS_V0, TS_V1, TS_V2, TS_V3 };
enum { TI_ACT = 0, TI_BUSY, TI_CH, TI_NJ, TI_J0, TI_J1, TI_J2, TI_J3, TI_J4, TI_J5, TI_J6, TI_J7,
       TI_J8, TI_J9, TI_J10, TI_J11 };

// --------------------------------------------------------------------------------------
// Per-trajectory block reduction: every thread holds NV partial sums of its trajectory
// (tau = tid % T); sums over lanes of equal tau by shuffles, then over warps in a fixed
// order.  Result in out[tau*NV + v].  Deterministic (FP64 throughout).
// For NV a power of two the first shuffle levels transpose: at offset o a lane sends half of its
// live values to its partner and adds the partner's other half, so each level halves the live
// values (8 values over 5 levels: 9 additions per lane instead of 40 -- FP64 runs at 1/64 of the
// FP32 rate on this GPU).  Slot q of lane l then holds value q + idx(l), idx from the lane bits of
// the transposing levels; the remaining levels add plainly.
template <int NV>
__device__ __forceinline__ void reduce_tau(double (&v)[NV], const KtGeom &g, double *red, double *out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int o = 16, live = NV, idx = 0, tmask = 0;
  if constexpr (NV > 1 && (NV & (NV - 1)) == 0) {
#pragma unroll
    for (int h = NV / 2; h >= 1; h >>= 1) {
      if (o >= g.T) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < h; ++q) {
          const double send = up ? v[q] : v[q + h];
          const double keep = up ? v[q + h] : v[q];
          v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
        if (up) idx += h;
        tmask |= o;
        live = h;
        o >>= 1;
      }
    }
  }
  for (; o >= g.T; o >>= 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q < live) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  if (((lane & ~(g.T - 1)) & ~tmask) == 0) {
    const int tau = lane & (g.T - 1);
#pragma unroll
    for (int q = 0; q < NV; ++q)
      if (q < live) red[(warp * g.T + tau) * 8 + q + idx] = v[q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < g.T * NV; t += blockDim.x) {
    const int tau = t / NV, q = t % NV;
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) s += red[(w * g.T + tau) * 8 + q];
    out[tau * NV + q] = s;
  }
  __syncthreads();
}

// --------------------------------------------------------------------------------------
// Per-interval tables: generator factors for pulse eps (scaled by 1/r, diagonal shifted),
// plus control factors for the update overlap.
template <typename R>
// pulse_only: the tables of a later interval of a whole sweep -- only the entries that depend on the
// pulse (node factors, diagonal, the last node's dense factor) are rebuilt, the rest is unchanged.
__device__ void build_tables(const KtGeom &g, const KtGenImage &im, const KtOps &ops, const Smem &sm,
                             const double *eps, bool with_hc, bool pulse_only = false) {
  typedef typename C2<R>::T C;
  C *lv = (C *)sm.loc_val;
  C *dg = (C *)sm.diag;
  C *pv = (C *)sm.pair_val;
  const int nls = g.n_loc * g.S;
  for (int e = threadIdx.x; e < g.n_nodes * nls; e += blockDim.x) {
    const int i = e / nls, rem = e % nls;
    double re = im.loc_base[e].re, imv = im.loc_base[e].im;
    for (int t = 0; t < g.n_cterms; ++t)
      if (g.cterm_node[t] == i) {
        re += eps[g.cterm_ctrl[t]] * im.ctrl_slot[t * nls + rem].re;
        imv += eps[g.cterm_ctrl[t]] * im.ctrl_slot[t * nls + rem].im;
      }
    lv[e] = mkc((R)re, (R)imv);
    if (!pulse_only) sm.loc_off[e] = im.loc_dl[e] * g.stride[i] * g.T;
  }
  for (int e = threadIdx.x; e < g.n_nodes * g.n_loc; e += blockDim.x) {
    const int i = e / g.n_loc, x = e % g.n_loc;
    double re = im.diag_base[e].re, imv = im.diag_base[e].im;
    for (int t = 0; t < g.n_cterms; ++t)
      if (g.cterm_node[t] == i) {
        re += eps[g.cterm_ctrl[t]] * im.ctrl_diag[t * g.n_loc + x].re;
        imv += eps[g.cterm_ctrl[t]] * im.ctrl_diag[t * g.n_loc + x].im;
      }
    dg[e] = mkc((R)re, (R)imv);
  }
  const int nl2 = g.n_loc * g.n_loc;
  if (!pulse_only)
    for (int e = threadIdx.x; e < g.n_pairs * nl2; e += blockDim.x) {
      sm.pair_off[e] = im.pair_off[e] * g.T;
      pv[e] = from_kc<C>(im.pair_val[e]);
    }
  {
    // last node's factor as a dense n_loc x n_loc table, ladder values, pair coefficients
    C *ld = (C *)sm.ldense;
    C *lr = (C *)sm.lora;
    C *pc = (C *)sm.pcoef;
    const int last = g.n_nodes - 1;
    for (int e = threadIdx.x; e < g.n_loc * g.n_loc; e += blockDim.x) ld[e] = mkc((R)0, (R)0);
    if (!pulse_only) {
      for (int e = threadIdx.x; e < g.n_loc; e += blockDim.x) {
        lr[e] = from_kc<C>(ops.lo_val[e]);
        lr[g.n_loc + e] = from_kc<C>(ops.ra_val[e]);
      }
      for (int e = threadIdx.x; e < g.n_pairs; e += blockDim.x) pc[e] = from_kc<C>(im.pair_coef[e]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < g.n_loc * g.S; e += blockDim.x) {
      const int idx = last * nls + e, x = e / g.S, dl = im.loc_dl[idx];
      if (dl) ld[x * g.n_loc + x + dl] = lv[idx];
    }
  }
  if (with_hc && !pulse_only) {
    C *hv = (C *)sm.hc_val;
    const int nh = g.n_loc * g.SH;
    for (int e = threadIdx.x; e < g.n_cterms * nh; e += blockDim.x) {
      const int t = e / nh;
      sm.hc_off[e] = ops.hc_dl[e] * g.stride[g.cterm_node[t]] * g.T;
      hv[e] = from_kc<C>(ops.hc_val[e]);
    }
  }
}

// Scaled generator Ghat applied at one item (element x, trajectory tau) of tile vector v.
template <typename R>
__device__ __forceinline__ typename C2<R>::T apply_item(const KtGeom &g, const KtGenImage &im, const Smem &sm,
                                                        const typename C2<R>::T *__restrict__ v,
                                                        int item, uint32_t dig,
                                                        typename C2<R>::T dval) {
  typedef typename C2<R>::T C;
  const C *lv = (const C *)sm.loc_val;
  const C *pv = (const C *)sm.pair_val;
  C out = cmul(dval, v[item]);
  for (int i = 0; i < g.n_nodes; ++i) {
    const int xi = (dig >> (4 * i)) & 15;
    const int base = (i * g.n_loc + xi) * g.S;
    for (int s = 0; s < g.S; ++s) {
      const int off = sm.loc_off[base + s];
      if (off) out = cfma(lv[base + s], v[item + off], out);
    }
  }
  const int nl2 = g.n_loc * g.n_loc;
  for (int p = 0; p < g.n_pairs; ++p) {
    const int xd = (dig >> (4 * im.pair_dst[p])) & 15;
    const int xs = (dig >> (4 * im.pair_src[p])) & 15;
    const int idx = p * nl2 + xd * g.n_loc + xs;
    const int off = sm.pair_off[idx];
    if (off) out = cfma(pv[idx], v[item + off], out);
  }
  return out;
}

template <typename R>
__device__ __forceinline__ typename C2<R>::T diag_of(const KtGeom &g, const Smem &sm, uint32_t dig) {
  typedef typename C2<R>::T C;
  const C *dg = (const C *)sm.diag;
  C s = mkc((R)0, (R)0);
  for (int i = 0; i < g.n_nodes; ++i) {
    const C v = dg[i * g.n_loc + ((dig >> (4 * i)) & 15)];
    s.x += v.x;
    s.y += v.y;
  }
  return s;
}

// Items of this thread: item_q = tid + q * nthreads, valid while < d*T.
template <int EPT, bool FIBER>
struct ItemsT {
  // strided mapping: item_q = tid + q * nthreads
  int item_[EPT];
  uint32_t dig_[EPT];
  bool ok_[EPT];
  __device__ __forceinline__ int item(int q) const { return item_[q]; }
  __device__ __forceinline__ uint32_t dig(int q) const { return dig_[q]; }
  __device__ __forceinline__ bool ok(int q) const { return ok_[q]; }
};
template <int EPT>
struct ItemsT<EPT, true> {
  // fiber mapping: the thread's items run along the last node's digit, so everything follows
  // from the first item, the fiber's digits (last digit 0) and the tile width
  int base, T, shift;
  uint32_t fdig;
  bool okf;
  __device__ __forceinline__ int item(int q) const { return base + q * T; }
  __device__ __forceinline__ uint32_t dig(int q) const { return fdig + ((uint32_t)q << shift); }
  __device__ __forceinline__ bool ok(int) const { return okf; }
};
template <int EPT, int NL>
using Items = ItemsT<EPT, (NL > 0)>;

template <int EPT, int NL>
__device__ __forceinline__ void load_items(const KtGeom &g, const KtOps &ops, Items<EPT, NL> &it) {
  if constexpr (NL > 0) {
    // fiber mapping: thread -> (fiber f, trajectory tau); its NL items run along the last
    // node's digit (stride T in the interleaved tile), so node-local and pair coefficients of
    // the other nodes are fixed per thread and the last node's are uniform per item slot
    const int f = threadIdx.x / g.T, tau = threadIdx.x % g.T;
    it.okf = f < g.d / NL;
    it.base = f * NL * g.T + tau;
    it.T = g.T;
    it.shift = 4 * (g.n_nodes - 1);
    it.fdig = it.okf ? ops.digits[f * NL] : 0u;
  } else {
    const int n = g.d * g.T;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int item = threadIdx.x + q * blockDim.x;
      it.item_[q] = item;
      it.ok_[q] = item < n;
      it.dig_[q] = it.ok_[q] ? ops.digits[item / g.T] : 0u;
    }
  }
}

// Ghat applied to the whole fiber of this thread: out[q] = (Ghat v)[item_q], q < NL.
// Coefficients of nodes other than the last are looked up once per fiber; those of the last
// node depend only on q and are the same for every lane.
template <typename R, int NL>
__device__ __forceinline__ void apply_fiber(const KtGeom &g, const KtGenImage &im, const Smem &sm,
                                            const typename C2<R>::T *__restrict__ v, int base, uint32_t fdig,
                                            typename C2<R>::T Df, typename C2<R>::T (&out)[NL]) {
  typedef typename C2<R>::T C;
  const C *lv = (const C *)sm.loc_val;
  const C *pv = (const C *)sm.pair_val;
  const C *dg = (const C *)sm.diag;
  const int last = g.n_nodes - 1;
  const int T = g.T;
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    const C dq = dg[last * NL + q];
    out[q] = cmul(mkc(Df.x + dq.x, Df.y + dq.y), v[base + q * T]);
  }
  // last node: row q of its factor
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    const int e0 = (last * NL + q) * g.S;
    for (int s = 0; s < g.S; ++s) {
      const int off = sm.loc_off[e0 + s];
      if (off) out[q] = cfma(lv[e0 + s], v[base + q * T + off], out[q]);
    }
  }
  // other nodes: one row per fiber
  for (int i = 0; i < last; ++i) {
    const int e0 = (i * NL + ((fdig >> (4 * i)) & 15)) * g.S;
    for (int s = 0; s < g.S; ++s) {
      const int off = sm.loc_off[e0 + s];
      if (off) {
        const C w = lv[e0 + s];
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = cfma(w, v[base + q * T + off], out[q]);
      }
    }
  }
  // pair hops a_dst^dag a_src
  for (int p = 0; p < g.n_pairs; ++p) {
    const int pd = im.pair_dst[p], ps = im.pair_src[p];
    const int pb = p * NL * NL;
    if (pd != last && ps != last) {
      const int e = pb + ((fdig >> (4 * pd)) & 15) * NL + ((fdig >> (4 * ps)) & 15);
      const int off = sm.pair_off[e];
      if (off) {
        const C w = pv[e];
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = cfma(w, v[base + q * T + off], out[q]);
      }
    } else if (pd == last) {
      const int e0 = pb + ((fdig >> (4 * ps)) & 15);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const int off = sm.pair_off[e0 + q * NL];
        if (off) out[q] = cfma(pv[e0 + q * NL], v[base + q * T + off], out[q]);
      }
    } else {
      const int e0 = pb + ((fdig >> (4 * pd)) & 15) * NL;
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const int off = sm.pair_off[e0 + q];
        if (off) out[q] = cfma(pv[e0 + q], v[base + q * T + off], out[q]);
      }
    }
  }
}

// Chebyshev sum in fiber mapping (see cheb_run).
template <typename R, int NL, class IT>
__device__ void cheb_run_fiber(const KtGeom &g, const KtGenImage &im, const Smem &sm, const IT &it, int K,
                               typename C2<R>::T (&acc)[NL]) {
  typedef typename C2<R>::T C;
  C *A = (C *)sm.bufA;
  C *B = (C *)sm.bufB;
  const C *cf = (const C *)sm.coef;
  const C *dg = (const C *)sm.diag;
  const int tau = threadIdx.x % g.T;
  const bool ok = it.ok(0);
  const int base = it.item(0);
  const uint32_t fdig = it.dig(0);
  const int last = g.n_nodes - 1;
  C Df = mkc((R)0, (R)0);
  for (int i = 0; i < last; ++i) {
    const C v = dg[i * NL + ((fdig >> (4 * i)) & 15)];
    Df.x += v.x;
    Df.y += v.y;
  }
  const C c0 = cf[tau];
#pragma unroll
  for (int q = 0; q < NL; ++q) acc[q] = ok ? cmul(c0, A[base + q * g.T]) : mkc((R)0, (R)0);
  if (K == 1) { __syncthreads(); return; }
  C t[NL];
  if (ok) {
    apply_fiber<R, NL>(g, im, sm, A, base, fdig, Df, t);
    const C c1 = cf[g.T + tau];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      B[base + q * g.T] = t[q];
      acc[q] = cfma(c1, t[q], acc[q]);
    }
  }
  __syncthreads();
  C *P = A;   // holds T_{k-1}; receives T_{k+1}
  C *Q = B;   // holds T_k
  for (int k = 2; k < K; ++k) {
    if (ok) {
      const C a = cf[k * g.T + tau];
      apply_fiber<R, NL>(g, im, sm, Q, base, fdig, Df, t);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const C old = P[base + q * g.T];
        const C nv = mkc(t[q].x + t[q].x - old.x, t[q].y + t[q].y - old.y);
        P[base + q * g.T] = nv;
        acc[q] = cfma(a, nv, acc[q]);
      }
    }
    __syncthreads();
    C *tmp = P; P = Q; Q = tmp;
  }
}

// Chebyshev sum: acc = sum_k coef[k][tau] T_k(Ghat) v with v in A on entry (synced).
// A and B are overwritten.  Ends synchronised.
template <typename R, int EPT, class IT>
__device__ void cheb_run(const KtGeom &g, const KtGenImage &im, const Smem &sm, const IT &it, int K,
                         typename C2<R>::T (&acc)[EPT]) {
  typedef typename C2<R>::T C;
  C *A = (C *)sm.bufA;
  C *B = (C *)sm.bufB;
  const C *cf = (const C *)sm.coef;
  const int tau = threadIdx.x % g.T;
  C dv[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    dv[q] = it.ok(q) ? diag_of<R>(g, sm, it.dig(q)) : mkc((R)0, (R)0);
    acc[q] = it.ok(q) ? cmul(cf[tau], A[it.item(q)]) : mkc((R)0, (R)0);
  }
  if (K == 1) { __syncthreads(); return; }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    if (!it.ok(q)) continue;
    const C t = apply_item<R>(g, im, sm, A, it.item(q), it.dig(q), dv[q]);
    B[it.item(q)] = t;
    acc[q] = cfma(cf[g.T + tau], t, acc[q]);
  }
  __syncthreads();
  C *P = A;   // holds T_{k-1}; receives T_{k+1}
  C *Q = B;   // holds T_k
  for (int k = 2; k < K; ++k) {
    const C a = cf[k * g.T + tau];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (!it.ok(q)) continue;
      const C t = apply_item<R>(g, im, sm, Q, it.item(q), it.dig(q), dv[q]);
      const C old = P[it.item(q)];
      const C nv = mkc(t.x + t.x - old.x, t.y + t.y - old.y);
      P[it.item(q)] = nv;
      acc[q] = cfma(a, nv, acc[q]);
    }
    __syncthreads();
    C *tmp = P; P = Q; Q = tmp;
  }
}

// Coefficients of exp(-i G s) for trajectory tau (called by one thread per trajectory):
// (2 - delta_k0) (-i)^k J_k(r s) exp(-i c s).
template <typename R>
__device__ void tau_coefs(const KtGeom &g, const Smem &sm, int tau, double c_gen, double s) {
  typedef typename C2<R>::T C;
  C *cf = (C *)sm.coef;
  double J[KT_MAX_K];
  kt_bessel_miller(g.r * s, g.K, J);
  double sn, cs;
  sincos(-c_gen * s, &sn, &cs);
  for (int k = 0; k < g.K; ++k) {
    const double m = (k == 0 ? 1.0 : 2.0) * J[k];
    double re, im;                           // m * (-i)^k
    switch (k & 3) {
      case 0: re = m; im = 0; break;
      case 1: re = 0; im = -m; break;
      case 2: re = -m; im = 0; break;
      default: re = 0; im = m; break;
    }
    cf[k * g.T + tau] = mkc((R)(re * cs - im * sn), (R)(re * sn + im * cs));
  }
}

template <typename R>
__device__ void uniform_coefs(const KtGeom &g, const Smem &sm, const KtCplx *full) {
  typedef typename C2<R>::T C;
  C *cf = (C *)sm.coef;
  for (int e = threadIdx.x; e < g.K * g.T; e += blockDim.x) cf[e] = from_kc<C>(full[e / g.T]);
}

template <typename R, int EPT, class IT>
__device__ __forceinline__ void load_tile(const KtGeom &g, const IT &it, const typename C2<R>::T *src,
                                          typename C2<R>::T *dst) {
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (it.ok(q)) dst[it.item(q)] = src[it.item(q)];
}

// Norm^2 of each trajectory of acc -> sm.tsc[TS_NRM][tau]
template <typename R, int EPT, class IT>
__device__ void norms(const KtGeom &g, const Smem &sm, const IT &it, const typename C2<R>::T (&acc)[EPT]) {
  R s = 0;
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (it.ok(q)) s += acc[q].x * acc[q].x + acc[q].y * acc[q].y;
  double v[1] = {(double)s};
  reduce_tau<1>(v, g, sm.red, sm.tsc + TS_NRM * g.T);
}

// (sum_i coef_i a_i) v  (adj = 0)  or  (sum_i conj(coef_i) a_i^dag) v  (adj = 1) at one item.
template <typename R>
__device__ __forceinline__ typename C2<R>::T lind_item(const KtGeom &g, const KtOps &ops, int l, int adj,
                                                       const typename C2<R>::T *v, int item, uint32_t dig) {
  typedef typename C2<R>::T C;
  C out = mkc((R)0, (R)0);
  for (int i = 0; i < g.n_nodes; ++i) {
    const int xi = (dig >> (4 * i)) & 15;
    KtCplx lc = ops.lind_coef[l * g.n_nodes + i];
    KtCplx av = adj ? ops.ra_val[xi] : ops.lo_val[xi];
    const int dl = adj ? ops.ra_dl[xi] : ops.lo_dl[xi];
    if (av.re == 0.0 && av.im == 0.0) continue;
    if (lc.re == 0.0 && lc.im == 0.0) continue;
    if (adj) lc.im = -lc.im;
    const double wr = lc.re * av.re - lc.im * av.im, wi = lc.re * av.im + lc.im * av.re;
    out = cfma(mkc((R)wr, (R)wi), v[item + dl * g.stride[i] * g.T], out);
  }
  return out;
}

// --------------------------------------------------------------------------------------
// Cavity-structure fast path.  Valid when every node is a three-level atom {g, e, r} times a
// cavity with photon numbers 0..NC (local index atom * (NC+1) + n), the ladder factor is the
// cavity annihilation operator, and the last node's factor couples only (r, n-1) <-> (g, n)
// (cavity) and (r, n) <-> (e, n) (drive) besides its diagonal -- the node of Sec. 3.1.  Then
// every coupling inside a thread's fiber (which runs over the last node) has a position known
// at compile time: the fiber's own T_k stays in registers and the last node's factor and the
// pair hops that raise or lower its photon number become register-indexed FMAs.
// The fiber's rows of the other nodes' factors (at most three other nodes on the fiber path: the
// fiber of the last node holds n_loc^(N-1) <= 736 threads' worth of the tile), loaded once per
// Chebyshev series: element offsets of the real and imaginary slot and their coefficients.
template <typename R>
struct RowCache {
  int off0[3], off1[3];
  R a[3], b[3];
};

template <typename R, int NL>
__device__ __forceinline__ void load_rows(const KtGeom &g, const Smem &sm, uint32_t fdig, RowCache<R> &rc) {
  typedef typename C2<R>::T C;
  const C *lv = (const C *)sm.loc_val;
  const int last = g.n_nodes - 1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    rc.off0[i] = rc.off1[i] = 0;
    rc.a[i] = rc.b[i] = (R)0;
    if (i < last) {
      const int e0 = (i * NL + ((fdig >> (4 * i)) & 15)) * 2;
      rc.off0[i] = sm.loc_off[e0];
      rc.off1[i] = sm.loc_off[e0 + 1];
      rc.a[i] = lv[e0].x;
      rc.b[i] = lv[e0 + 1].y;
    }
  }
}

// Constants of the real / imaginary kernels (kernel parameters of the image, see KtGenImage).
template <typename R> __device__ __forceinline__ const R *acs_kd(const KtGenImage &im);
template <> __device__ __forceinline__ const float *acs_kd<float>(const KtGenImage &im) { return im.kd32; }
template <> __device__ __forceinline__ const double *acs_kd<double>(const KtGenImage &im) { return im.kd64; }
template <typename R> __device__ __forceinline__ const R *acs_kc(const KtGenImage &im);
template <> __device__ __forceinline__ const float *acs_kc<float>(const KtGenImage &im) { return im.kc32; }
template <> __device__ __forceinline__ const double *acs_kc<double>(const KtGenImage &im) { return im.kc64; }
template <typename R> __device__ __forceinline__ const R *acs_kp(const KtGenImage &im);
template <> __device__ __forceinline__ const float *acs_kp<float>(const KtGenImage &im) { return im.kp32; }
template <> __device__ __forceinline__ const double *acs_kp<double>(const KtGenImage &im) { return im.kp64; }
// sqrt(n) for the photon numbers n <= 2 of the cavity-structure node (<n-1|a|n>; the host has
// checked that the ladder factor holds exactly these values)
template <typename R>
__device__ __forceinline__ R sqrt_n(int n) {
  return n >= 2 ? (R)1.4142135623730951 : (n == 1 ? (R)1 : (R)0);
}

// RI: the couplings are purely real or imaginary by class (host check: node rows hold
// [real, imaginary] slots, last-node cavity real and drive imaginary, pair coefficients imaginary,
// ladder values sqrt(n), no control on the last node's diagonal or cavity couplings), applied with
// two FMAs each; the pulse-independent coefficients (last node's diagonal and cavity couplings,
// pair coefficients, ladder values) are kernel-parameter or compile-time constants, so only the
// drive couplings, the other nodes' pair tables and the states are read from shared memory.
// CACHE: the other nodes' rows come from rc (registers) instead of the shared tables.
template <typename R, int NC, int TT, bool RI, bool CACHE>
__device__ __forceinline__ void apply_acs(const KtGeom &g, const KtGenImage &im, const Smem &sm,
                                          const typename C2<R>::T *__restrict__ v, int base, uint32_t fdig,
                                          typename C2<R>::T Df, const typename C2<R>::T (&vk)[3 * (NC + 1)],
                                          typename C2<R>::T (&out)[3 * (NC + 1)], const RowCache<R> &rc) {
  typedef typename C2<R>::T C;
  constexpr int NP = NC + 1, NL = 3 * NP;
  const C *lv = (const C *)sm.loc_val;
  const C *pv = (const C *)sm.pair_val;
  const C *dg = (const C *)sm.diag;
  const C *ld = (const C *)sm.ldense;
  const C *lo = (const C *)sm.lora;
  const C *ra = lo + NL;
  const C *pc = (const C *)sm.pcoef;
  const int last = g.n_nodes - 1;
  const int T = TT > 0 ? TT : g.T;   // TT > 0: tile width fixed at compile time
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    C dq;
    if constexpr (RI) dq = mkc(acs_kd<R>(im)[2 * q], acs_kd<R>(im)[2 * q + 1]);
    else dq = dg[last * NL + q];
    out[q] = cmul(mkc(Df.x + dq.x, Df.y + dq.y), vk[q]);
  }
  // last node: cavity (r, n-1) <-> (g, n) and drive (r, n) <-> (e, n)
#pragma unroll
  for (int n = 1; n <= NC; ++n) {
    const int qr = 2 * NP + n - 1, qg = n;
    if constexpr (RI) {
      out[qr] = rfma(acs_kc<R>(im)[n - 1], vk[qg], out[qr]);
      out[qg] = rfma(acs_kc<R>(im)[NC + n - 1], vk[qr], out[qg]);
    } else {
      out[qr] = cfma(ld[qr * NL + qg], vk[qg], out[qr]);
      out[qg] = cfma(ld[qg * NL + qr], vk[qr], out[qg]);
    }
  }
#pragma unroll
  for (int n = 0; n <= NC; ++n) {
    const int qr = 2 * NP + n, qe = NP + n;
    if constexpr (RI) {
      out[qr] = ifma(ld[qr * NL + qe].y, vk[qe], out[qr]);
      out[qe] = ifma(ld[qe * NL + qr].y, vk[qr], out[qe]);
    } else {
      out[qr] = cfma(ld[qr * NL + qe], vk[qe], out[qr]);
      out[qe] = cfma(ld[qe * NL + qr], vk[qr], out[qe]);
    }
  }
  // other nodes: one row per fiber, each entry one neighbouring fiber
  if constexpr (RI && !CACHE) {
    for (int i = 0; i < last; ++i) {
      const int e0 = (i * NL + ((fdig >> (4 * i)) & 15)) * 2;
      const int off0 = sm.loc_off[e0], off1 = sm.loc_off[e0 + 1];
      if (off0) {
        const R a = lv[e0].x;
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = rfma(a, v[base + off0 + q * T], out[q]);
      }
      if (off1) {
        const R b = lv[e0 + 1].y;
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = ifma(b, v[base + off1 + q * T], out[q]);
      }
    }
  } else if constexpr (RI) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (rc.off0[i]) {
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = rfma(rc.a[i], v[base + rc.off0[i] + q * T], out[q]);
      }
      if (rc.off1[i]) {
#pragma unroll
        for (int q = 0; q < NL; ++q) out[q] = ifma(rc.b[i], v[base + rc.off1[i] + q * T], out[q]);
      }
    }
  } else {
    for (int i = 0; i < last; ++i) {
      const int e0 = (i * NL + ((fdig >> (4 * i)) & 15)) * g.S;
      for (int s = 0; s < g.S; ++s) {
        const int off = sm.loc_off[e0 + s];
        if (off) {
          const C w = lv[e0 + s];
#pragma unroll
          for (int q = 0; q < NL; ++q) out[q] = cfma(w, v[base + off + q * T], out[q]);
        }
      }
    }
  }
  // pair hops coef a_dst^dag a_src
  for (int p = 0; p < g.n_pairs; ++p) {
    const int pd = im.pair_dst[p], ps = im.pair_src[p];
    if (pd != last && ps != last) {
      const int e = p * NL * NL + ((fdig >> (4 * pd)) & 15) * NL + ((fdig >> (4 * ps)) & 15);
      const int off = sm.pair_off[e];
      if (off) {
        if constexpr (RI) {
          const R b = pv[e].y;
#pragma unroll
          for (int q = 0; q < NL; ++q) out[q] = ifma(b, v[base + off + q * T], out[q]);
        } else {
          const C w = pv[e];
#pragma unroll
          for (int q = 0; q < NL; ++q) out[q] = cfma(w, v[base + off + q * T], out[q]);
        }
      }
    } else if (pd == last) {
      // raise the last node (q <- q-1, n_q >= 1), lower node ps (x_s -> x_s + 1, n_s < NC)
      const int xs = (fdig >> (4 * ps)) & 15;
      if (xs % NP < NC) {
        const int off = g.stride[ps] * T;
        if constexpr (RI) {
          const R cb = acs_kp<R>(im)[p] * sqrt_n<R>(xs % NP + 1);
#pragma unroll
          for (int q = 0; q < NL; ++q) {
            if (q % NP == 0) continue;
            out[q] = ifma(cb * sqrt_n<R>(q % NP), v[base + off + (q - 1) * T], out[q]);
          }
        } else {
          const C cf = cmul(pc[p], lo[xs]);
#pragma unroll
          for (int q = 0; q < NL; ++q) {
            if (q % NP == 0) continue;
            out[q] = cfma(cmul(cf, ra[q]), v[base + off + (q - 1) * T], out[q]);
          }
        }
      }
    } else {
      // lower the last node (q <- q+1, n_q < NC), raise node pd (x_d -> x_d - 1, n_d >= 1)
      const int xd = (fdig >> (4 * pd)) & 15;
      if (xd % NP >= 1) {
        const int off = -g.stride[pd] * T;
        if constexpr (RI) {
          const R cb = acs_kp<R>(im)[p] * sqrt_n<R>(xd % NP);
#pragma unroll
          for (int q = 0; q < NL; ++q) {
            if (q % NP == NC) continue;
            out[q] = ifma(cb * sqrt_n<R>(q % NP + 1), v[base + off + (q + 1) * T], out[q]);
          }
        } else {
          const C cf = cmul(pc[p], ra[xd]);
#pragma unroll
          for (int q = 0; q < NL; ++q) {
            if (q % NP == NC) continue;
            out[q] = cfma(cmul(cf, lo[q]), v[base + off + (q + 1) * T], out[q]);
          }
        }
      }
    }
  }
}

template <typename R, int NC, int TT, bool RI, bool CACHE, class IT>
__device__ void cheb_run_acs(const KtGeom &g, const KtGenImage &im, const Smem &sm, const IT &it,
                             int K, typename C2<R>::T (&acc)[3 * (NC + 1)]) {
  typedef typename C2<R>::T C;
  constexpr int NL = 3 * (NC + 1);
  C *A = (C *)sm.bufA;
  C *B = (C *)sm.bufB;
  const C *cf = (const C *)sm.coef;
  const C *dg = (const C *)sm.diag;
  const int T = TT > 0 ? TT : g.T;
  const int tau = TT == 1 ? 0 : (int)(threadIdx.x % T);
  const bool ok = it.ok(0);
  const int base = it.item(0);
  const uint32_t fdig = it.dig(0);
  const int last = g.n_nodes - 1;
  C Df = mkc((R)0, (R)0);
  for (int i = 0; i < last; ++i) {
    const C v = dg[i * NL + ((fdig >> (4 * i)) & 15)];
    Df.x += v.x;
    Df.y += v.y;
  }
  RowCache<R> rc;
  if constexpr (RI && CACHE) {
    if (ok) load_rows<R, NL>(g, sm, fdig, rc);
  }
  C vk[NL];
  const C c0 = cf[tau];
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    vk[q] = ok ? A[base + q * T] : mkc((R)0, (R)0);
    acc[q] = cmul(c0, vk[q]);
  }
  if (K == 1) { __syncthreads(); return; }
  C t[NL];
  if (ok) {
    apply_acs<R, NC, TT, RI, CACHE>(g, im, sm, A, base, fdig, Df, vk, t, rc);
    const C c1 = cf[T + tau];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      B[base + q * T] = t[q];
      acc[q] = cfma(c1, t[q], acc[q]);
      vk[q] = t[q];
    }
  }
  __syncthreads();
  C *P = A;   // holds T_{k-1}; receives T_{k+1}
  C *Q = B;   // holds T_k (this thread's fiber also in vk)
  for (int k = 2; k < K; ++k) {
    if (ok) {
      const C a = cf[k * T + tau];
      apply_acs<R, NC, TT, RI, CACHE>(g, im, sm, Q, base, fdig, Df, vk, t, rc);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const C old = P[base + q * T];
        const C nv = mkc(t[q].x + t[q].x - old.x, t[q].y + t[q].y - old.y);
        P[base + q * T] = nv;
        acc[q] = cfma(a, nv, acc[q]);
        vk[q] = nv;
      }
    }
    __syncthreads();
    C *tmp = P; P = Q; Q = tmp;
  }
}

template <typename R, int EPT, int NL, int ACS, bool CACHE, class IT>
__device__ __forceinline__ void cheb_dispatch(const KtGeom &g, const KtGenImage &im, const Smem &sm,
                                              const IT &it, int K, typename C2<R>::T (&acc)[EPT]) {
  // ACS: 1 cavity structure, 2 the same with T = 1, 3 with real / imaginary couplings, 4 both
  if constexpr (ACS) cheb_run_acs<R, NL / 3 - 1, (ACS == 2 || ACS == 4) ? 1 : 0, (ACS >= 3), CACHE>(g, im, sm, it, K, acc);
  else if constexpr (NL > 0) cheb_run_fiber<R, NL>(g, im, sm, it, K, acc);
  else cheb_run<R, EPT>(g, im, sm, it, K, acc);
}

// End of a tile in the forward kernel looping over tiles: the generic-proxy writes of the tile are
// ordered before the bulk copies that will overwrite its buffers, then the prefetched psi (fourth
// buffer) becomes the next tile's input and the old input buffer (maybe still being stored) the next
// prefetch target.
__device__ __forceinline__ void end_fwd_tile(Smem &sm, bool persist) {
  if (!persist) return;
  fence_proxy_async_smem();
  __syncthreads();
  void *t = sm.bufA;
  sm.bufA = sm.bufD;
  sm.bufD = t;
}

// --------------------------------------------------------------------------------------
// Forward interval kernel.  One Chebyshev call site serves every phase:
//   MAIN    full interval from psi(t_{j-1}) (uniform coefficients),
//   BISECT  bisection of ||exp(-i G s) start||^2 = r for flagged trajectories,
//   SSTAR   the state at the located jump time s*, then collapse (Sec. 2.1, steps 3-5),
//   REST    the remainder of the interval from the collapsed state, tested again.
enum { PH_MAIN = 0, PH_BISECT, PH_SSTAR, PH_REST, PH_DONE };

template <typename R, int EPT, int NL, int ACS, bool SWEEP>
__global__ void __launch_bounds__(NL > 0 ? 736 : (sizeof(R) == 8 ? 512 : 1024)) fwd_kernel(KtGeom g, KtGenImage im, KtOps ops, FwdArgs a) {
  typedef typename C2<R>::T C;
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm;
  // with g.fwd_grid > 0 the CTAs loop over tiles blockIdx.x, blockIdx.x + gridDim.x, ...: the tables and
  // the item mapping are built once, and the next tile's psi (fourth buffer, barriers [0] / [3] in turn)
  // and chi (third buffer) arrive by bulk copy while the current tile is propagated.
  // SWEEP (a.sweep): one cooperative launch runs intervals a.j .. nt of one tile per CTA (see FwdArgs);
  // a compile-time switch, so that the per-interval kernels carry none of the sweep's state.
  constexpr bool sweep = SWEEP;
  const bool persist = !sweep && g.fwd_grid > 0;
  carve(g, sizeof(C), smem_raw, &sm, g.prefetch_chi != 0, persist);
  const int tau = threadIdx.x % g.T;
  // bisection stop: 2^-48 dt in FP64 (near the rounding of the FP64 norm it compares), 2^-40 dt in
  // FP32-mixed (far below the FP32 norm's own error)
  const double tol = (sizeof(R) == 8 ? 0x1p-48 : 0x1p-40) * g.dt;
  int j = a.j;

  if (threadIdx.x < g.n_ctrl) {
    const int c = threadIdx.x;
    double e = 0.0;
    if (j >= 1) {
      e = a.eps_old[c * a.nt + (j - 1)];
      if (a.update) e += a.deps[c * a.nt + (j - 1)];
    }
    sm.eps[c] = e;
  }
  if (threadIdx.x < 8) sm.flag[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    mbar_init(&sm.mbar[0], 1);
    mbar_init(&sm.mbar[1], 1);
    mbar_init(&sm.mbar[2], 1);
    mbar_init(&sm.mbar[3], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t tile_bytes = (uint32_t)(g.tile_elems * sizeof(C));
  // co-states chi(t_i) of interval i's update overlap
  auto chi_of = [&](int i, int t) -> const C * {
    const C *base = sweep ? (const C *)((const char *)a.chi_slots + (size_t)i * a.slot_bytes) : (const C *)a.chi_t;
    return base + (size_t)t * g.tile_elems;
  };
  // the bulk engine brings psi(t_{j-1}) (and chi(t_j) when there is room) while the tables are built
  if (threadIdx.x == 0) {
    bulk_load(sm.bufA, (const C *)a.psi_in + (size_t)blockIdx.x * g.tile_elems, tile_bytes, &sm.mbar[0]);
    if (a.overlap && j < a.nt && g.prefetch_chi) bulk_load(sm.bufC, chi_of(j, blockIdx.x), tile_bytes, &sm.mbar[1]);
  }
  build_tables<R>(g, im, ops, sm, sm.eps, a.overlap != 0);
  Items<EPT, NL> it;
  load_items<EPT, NL>(g, ops, it);
  bool store_pending = false;
  unsigned nchi = 0;        // chi loads waited for on barrier [1] (the n-th completes phase n & 1)
  bool coef_full = false;   // the full-step coefficients are in place (no jump phase overwrote them)
  unsigned sync_gen = 0;    // grid barriers passed (sweep)
  C acc[EPT];
  for (;; ++j) {            // intervals: one unless sweep
    const bool need_chi = a.overlap && j < a.nt;
    // sweep: the update's pulse-independent factors for the finisher, read now, off its critical path
    // (the per-interval kernels read them in the finisher: registers held across the tiles spill there)
    double fin_scale = 0.0, fin_eold = 0.0;
    if (sweep && need_chi && threadIdx.x < g.n_ctrl) {
      const size_t idx = (size_t)threadIdx.x * a.nt + j;   // interval j+1 (0-based index j)
      fin_scale = a.shape[idx] / (g.lam[threadIdx.x] * g.M_norm);
      fin_eold = a.eps_old[idx];
    }
    if (j != a.j) {
      // sweep: the next interval.  Its pulse is in sm.eps (guess sweep: eps_old; updating: the value
      // the barrier's finisher formed), its chi goes to the third buffer once every thread is done
      // with the previous one, and the tables are rebuilt for the new pulse.
      if (!a.update && threadIdx.x < g.n_ctrl) sm.eps[threadIdx.x] = a.eps_old[threadIdx.x * a.nt + (j - 1)];
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0 && need_chi && g.prefetch_chi)
        bulk_load(sm.bufC, chi_of(j, blockIdx.x), tile_bytes, &sm.mbar[1]);
      build_tables<R>(g, im, ops, sm, sm.eps, a.overlap != 0, true);
    }
    int tile = blockIdx.x;
    for (int use = 0; tile < g.n_tiles; tile += gridDim.x, ++use) {
      const int next = tile + (int)gridDim.x;
      const C *psi_in = (const C *)((!sweep || j <= 1) ? a.psi_in : a.psi_ring[(j - 1) & 1]) + (size_t)tile * g.tile_elems;
      C *psi_out = (C *)(sweep ? a.psi_ring[j & 1] : a.psi_out) + (size_t)tile * g.tile_elems;
      const C *chi_g = need_chi ? chi_of(j, tile) : nullptr;
      // the trajectory's current threshold, read now so that its latency is off the path after the series
      const double r_start = (threadIdx.x < g.T) ? a.rstate[(size_t)tile * g.T + threadIdx.x] : 0.0;
      if (threadIdx.x == 0) {
        sm.flag[0] = 0;
        sm.flag[1] = 0;
        sm.flag[2] = 0;
      }
      C *A = (C *)sm.bufA;
      C *B = (C *)sm.bufB;
      if (sweep && j != a.j) {
        // sweep: psi(t_{j-1}) is the previous interval's result, still in registers
    #pragma unroll
        for (int q = 0; q < EPT; ++q)
          if (it.ok(q)) A[it.item(q)] = acc[q];
        __syncthreads();
      } else if (!tile_wait((use & 1) ? &sm.mbar[3] : &sm.mbar[0], (use >> 1) & 1, &sm.flag[4], a.status,
                            g.inject_timeout ? &sm.mbar[2] : nullptr)) {
        // psi of this tile: load number `use`, barrier [0] / [3] in turn, phase parity (use >> 1) & 1
        if (threadIdx.x == 0) {
          if (need_chi && g.prefetch_chi) mbar_wait_bounded(&sm.mbar[1], nchi & 1);
          if (store_pending) bulk_store_wait();
        }
        return;
      }
      if (persist && next < g.n_tiles) {
        // the fourth buffer fed the previous tile's bulk store: let that finish, then prefetch into it
        if (threadIdx.x == 0) {
          if (store_pending) bulk_store_wait();
          bulk_load(sm.bufD, (const C *)a.psi_in + (size_t)next * g.tile_elems, tile_bytes,
                    (use & 1) ? &sm.mbar[0] : &sm.mbar[3]);
        }
        store_pending = false;
      }
      bool jumped = false, stored = false;

      int phase = (j >= 1) ? PH_MAIN : PH_DONE;
      if (phase == PH_DONE) {
    #pragma unroll
        for (int q = 0; q < EPT; ++q) acc[q] = it.ok(q) ? A[it.item(q)] : mkc((R)0, (R)0);
      }
      int guard = 0;
      while (phase != PH_DONE) {
        // ---- choose the propagation of this round
        if (phase == PH_BISECT) {
          if (threadIdx.x == 0) sm.flag[1] = 0;
          __syncthreads();
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x;
            const double lo = sm.tsc[TS_LO * g.T + t], hi = sm.tsc[TS_HI * g.T + t];
            const int busy = sm.tin[TI_ACT * g.T + t] && (hi - lo > tol) && sm.tin[TI_CH * g.T + t] < 60;
            sm.tin[TI_BUSY * g.T + t] = busy;
            if (busy) atomicAdd(&sm.flag[1], 1);
          }
          __syncthreads();
          if (sm.flag[1] == 0) phase = PH_SSTAR;
        }
        if (phase == PH_MAIN) {
          // the full-step coefficients are the same for every interval: a sweep loads them once, again
          // only after a jump phase has overwritten them (the per-interval kernels reload them per tile:
          // skipping there costs them registers)
          if (!(sweep && coef_full)) uniform_coefs<R>(g, sm, im.cheb_full);
          coef_full = true;
        } else {
          coef_full = false;
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x;
            const bool act = sm.tin[TI_ACT * g.T + t] != 0;
            double len = 0.0;
            if (phase == PH_BISECT) len = sm.tin[TI_BUSY * g.T + t] ? 0.5 * (sm.tsc[TS_LO * g.T + t] + sm.tsc[TS_HI * g.T + t]) : 0.0;
            else if (phase == PH_SSTAR) len = act ? sm.tsc[TS_HI * g.T + t] : 0.0;
            else len = act ? g.dt - sm.tsc[TS_S0 * g.T + t] : 0.0;
            tau_coefs<R>(g, sm, t, g.c_fwd, len);
          }
        }
        if (phase != PH_MAIN) load_tile<R, EPT>(g, it, psi_out, A);   // the main round's tile came by bulk copy
        __syncthreads();
        cheb_dispatch<R, EPT, NL, ACS, true>(g, im, sm, it, g.K, acc);   // rows cached: measured faster here
        norms<R, EPT>(g, sm, it, acc);

        // ---- consume the result
        if (phase == PH_MAIN) {
    #pragma unroll
          for (int q = 0; q < EPT; ++q)
            if (it.ok(q)) A[it.item(q)] = acc[q];
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x, k = tile * g.T + t;
            const double nrm = sm.tsc[TS_NRM * g.T + t];
            const double r = r_start;                        // padding trajectories carry r = -1
            if (!isfinite(nrm)) set_status(a.status, KT_DEV_NONFINITE);
            const int act = (k < g.M) && (nrm <= r);         // jump iff ||psi||^2 <= r
            sm.tin[TI_ACT * g.T + t] = act;
            sm.tsc[TS_R * g.T + t] = r;
            sm.tsc[TS_S0 * g.T + t] = 0.0;
            // first-order scheme: the bracket starts closed at dt, the jump is applied at the end
            sm.tsc[TS_LO * g.T + t] = g.first_order ? g.dt : 0.0;
            sm.tsc[TS_HI * g.T + t] = g.dt;
            sm.tin[TI_CH * g.T + t] = 0;                     // bisection iteration counter
            if (act) atomicAdd(&sm.flag[0], 1);
          }
          __syncthreads();
          if (sm.flag[0] == 0) break;
          // a jump: the tile's results go to psi_out now (coalesced), and flagged trajectories
          // restart from psi(t_{j-1}), kept in psi_out
          jumped = true;
          for (int e = threadIdx.x; e < g.d * g.T; e += blockDim.x) psi_out[e] = A[e];
          __syncthreads();
    #pragma unroll
          for (int q = 0; q < EPT; ++q)
            if (it.ok(q) && sm.tin[TI_ACT * g.T + tau]) psi_out[it.item(q)] = psi_in[it.item(q)];
          __syncthreads();
          phase = PH_BISECT;
        } else if (phase == PH_BISECT) {
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x;
            if (sm.tin[TI_BUSY * g.T + t]) {
              const double mid = 0.5 * (sm.tsc[TS_LO * g.T + t] + sm.tsc[TS_HI * g.T + t]);
              if (sm.tsc[TS_NRM * g.T + t] <= sm.tsc[TS_R * g.T + t]) sm.tsc[TS_HI * g.T + t] = mid;
              else sm.tsc[TS_LO * g.T + t] = mid;
              sm.tin[TI_CH * g.T + t] += 1;
            }
          }
          __syncthreads();
        } else if (phase == PH_SSTAR) {
    #pragma unroll
          for (int q = 0; q < EPT; ++q)
            if (it.ok(q)) A[it.item(q)] = acc[q];
          __syncthreads();
          // channel probabilities p_l = ||L_l phi||^2
          double v[KT_MAX_LIND];
          for (int l = 0; l < KT_MAX_LIND; ++l) {
            R s = 0;
            if (l < g.n_lind) {
    #pragma unroll
              for (int q = 0; q < EPT; ++q)
                if (it.ok(q)) {
                  const C y = lind_item<R>(g, ops, l, 0, A, it.item(q), it.dig(q));
                  s += y.x * y.x + y.y * y.y;
                }
            }
            v[l] = (double)s;
          }
          reduce_tau<KT_MAX_LIND>(v, g, sm.red, sm.tsc + TS_V0 * g.T);
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x, k = tile * g.T + t;
            int ch = -1;
            if (sm.tin[TI_ACT * g.T + t]) {
              const double *p = sm.tsc + TS_V0 * g.T + t * KT_MAX_LIND;
              const int m = a.jcount[k] + 1;
              if (m > g.max_jumps) {
                set_status(a.status, KT_DEV_RECORD_FULL);
                sm.tin[TI_ACT * g.T + t] = 0;
              } else if (g.n_lind == 0) {
                set_status(a.status, KT_DEV_ZERO_JUMP);      // norm loss without any jump operator
                sm.tin[TI_ACT * g.T + t] = 0;
              } else {
                const double *U = a.U + ((size_t)*a.pass_row * g.M + k) * g.draws;
                double tot = 0.0;
                for (int l = 0; l < g.n_lind; ++l) tot += p[l];
                const double target = U[2 * m - 1] * tot;   // first channel whose cumulative p reaches u * sum p
                ch = g.n_lind - 1;
                double cum = 0.0;
                for (int l = 0; l < g.n_lind; ++l) {
                  cum += p[l];
                  if (cum >= target) { ch = l; break; }
                }
                if (!(p[ch] > 0.0)) {
                  set_status(a.status, KT_DEV_ZERO_JUMP);
                  sm.tin[TI_ACT * g.T + t] = 0;
                  ch = -1;
                } else {
                  const double cnorm = 1.0 / sqrt(p[ch]);
                  const double sstar = sm.tsc[TS_S0 * g.T + t] + sm.tsc[TS_HI * g.T + t];
                  const size_t ri = (size_t)k * g.max_jumps + (m - 1);
                  a.rec_step[ri] = j;
                  a.rec_ch[ri] = ch;
                  a.rec_s[ri] = sstar;
                  a.rec_c[ri] = cnorm;
                  a.jcount[k] = m;
                  const double rn = U[2 * m];
                  a.rstate[k] = rn;
                  sm.tsc[TS_R * g.T + t] = rn;
                  sm.tsc[TS_S0 * g.T + t] = sstar;
                  sm.tsc[TS_C * g.T + t] = cnorm;
                }
              }
            }
            sm.tin[TI_NJ * g.T + t] = ch;
          }
          __syncthreads();
          // collapse: start <- c L_ch phi
          const int ch = sm.tin[TI_NJ * g.T + tau];
          if (ch >= 0) {
            const R cn = (R)sm.tsc[TS_C * g.T + tau];
    #pragma unroll
            for (int q = 0; q < EPT; ++q) {
              if (!it.ok(q)) continue;
              const C y = lind_item<R>(g, ops, ch, 0, A, it.item(q), it.dig(q));
              psi_out[it.item(q)] = mkc(cn * y.x, cn * y.y);
            }
          }
          __syncthreads();
          phase = PH_REST;
        } else {  // PH_REST
          if (threadIdx.x == 0) sm.flag[2] = 0;
          __syncthreads();
          if (threadIdx.x < g.T) {
            const int t = threadIdx.x;
            int done = 0;
            if (sm.tin[TI_ACT * g.T + t]) {
              if (sm.tsc[TS_NRM * g.T + t] > sm.tsc[TS_R * g.T + t]) done = 1;
              else {
                atomicAdd(&sm.flag[2], 1);      // another jump inside the remainder
                sm.tsc[TS_HI * g.T + t] = g.dt - sm.tsc[TS_S0 * g.T + t];
                sm.tsc[TS_LO * g.T + t] = g.first_order ? sm.tsc[TS_HI * g.T + t] : 0.0;
                sm.tin[TI_CH * g.T + t] = 0;
              }
            }
            sm.tin[TI_BUSY * g.T + t] = done;
          }
          __syncthreads();
    #pragma unroll
          for (int q = 0; q < EPT; ++q)
            if (it.ok(q) && sm.tin[TI_BUSY * g.T + tau]) psi_out[it.item(q)] = acc[q];
          __syncthreads();
          if (threadIdx.x < g.T && sm.tin[TI_BUSY * g.T + threadIdx.x]) sm.tin[TI_ACT * g.T + threadIdx.x] = 0;
          __syncthreads();
          ++guard;
          if (sm.flag[2] == 0 || guard > g.max_jumps + 1) {
            // final states of the whole tile
    #pragma unroll
            for (int q = 0; q < EPT; ++q)
              if (it.ok(q)) acc[q] = psi_out[it.item(q)];
            __syncthreads();
            phase = PH_DONE;
          } else {
            phase = PH_BISECT;
          }
        }
      }

      if (j >= 1 && !jumped) {
        if (sweep) {
          // sweep: plain stores, read back by the next interval's jump restarts after a CTA barrier
    #pragma unroll
          for (int q = 0; q < EPT; ++q)
            if (it.ok(q)) psi_out[it.item(q)] = acc[q];
        } else {
          // psi(t_j) of the whole tile is in A: one bulk store to psi_out
          fence_proxy_async_smem();
          __syncthreads();
          if (threadIdx.x == 0) bulk_store(psi_out, A, tile_bytes);
          stored = true;
        }
      }

      // ---------------- end of the sweep: tau_k = <tgt|psi_k>/||psi_k|| ----------------
      if (j == a.nt) {
        double v[3] = {0.0, 0.0, 0.0};
    #pragma unroll
        for (int q = 0; q < EPT; ++q) {
          if (!it.ok(q)) continue;
          const KtCplx t = ops.tgt[it.item(q) / g.T];
          const double xr = (double)acc[q].x, xi = (double)acc[q].y;
          v[0] += t.re * xr + t.im * xi;   // conj(tgt) * psi
          v[1] += t.re * xi - t.im * xr;
          v[2] += xr * xr + xi * xi;
        }
        reduce_tau<3>(v, g, sm.red, sm.tsc + TS_V0 * g.T);
        if (threadIdx.x < g.T) {
          const int k = tile * g.T + threadIdx.x;
          const double *o = sm.tsc + TS_V0 * g.T + threadIdx.x * 3;
          const double nrm = o[2];
          // a trajectory's overlap is taken with the normalised state; a density matrix's
          // <<P_tgt|rho(T)>> is linear in rho and is not normalised
          const double inv = g.density ? 1.0 : (nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0);
          a.tau[k].re = o[0] * inv;
          a.tau[k].im = o[1] * inv;
          a.norm2[k] = nrm;
          if (!isfinite(nrm) || !isfinite(o[0]) || !isfinite(o[1])) set_status(a.status, KT_DEV_NONFINITE);
        }
        store_pending = store_pending || stored;
        end_fwd_tile(sm, persist);
        continue;
      }

      // ---------------- update overlap at t_j: g_c = sum_k Im <chi_k|hc_c|psi_k> ----------------
      if (!a.overlap) {
        store_pending = store_pending || stored;
        end_fwd_tile(sm, persist);
        continue;
      }
      if (jumped) {
        // final states came back through psi_out: put them into A for the neighbour reads
    #pragma unroll
        for (int q = 0; q < EPT; ++q)
          if (it.ok(q)) A[it.item(q)] = acc[q];
      }
      const C *chi;
      if (g.prefetch_chi) {
        chi = (const C *)sm.bufC;
      } else {
        // B was written by ordinary stores during the Chebyshev rounds: order them before the copy
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) bulk_load(B, chi_g, tile_bytes, &sm.mbar[1]);
        chi = B;
      }
      if (!tile_wait(&sm.mbar[1], nchi & 1, &sm.flag[5], a.status, g.inject_timeout ? &sm.mbar[2] : nullptr)) {
        if (threadIdx.x == 0) {
          if (store_pending || stored) bulk_store_wait();
          // the next tile's psi is on its way into the fourth buffer: let it land before leaving
          if (persist && next < g.n_tiles) mbar_wait_bounded((use & 1) ? &sm.mbar[0] : &sm.mbar[3], ((use + 1) >> 1) & 1);
        }
        return;
      }
      ++nchi;
      const C *hv = (const C *)sm.hc_val;
      // per-thread sums per control in the state precision (a trajectory problem has one term per
      // control; a density matrix a ket and a bra term), converted to FP64 once for the reduction
      R sc[KT_MAX_CTRL];
    #pragma unroll
      for (int c = 0; c < KT_MAX_CTRL; ++c) sc[c] = (R)0;
      for (int t = 0; t < g.n_cterms; ++t) {
        const int node = g.cterm_node[t];
        R s = 0;
        if (NL > 0 && node != g.n_nodes - 1) {
          // fiber mapping, control on another node: one factor row serves the whole fiber
          if (it.ok(0)) {
            const int base = (t * g.n_loc + ((it.dig(0) >> (4 * node)) & 15)) * g.SH;
            C h[EPT];
    #pragma unroll
            for (int q = 0; q < EPT; ++q) h[q] = mkc((R)0, (R)0);
            for (int e = 0; e < g.SH; ++e) {
              const C w = hv[base + e];
              if (w.x != (R)0 || w.y != (R)0) {
                const int off = sm.hc_off[base + e];
    #pragma unroll
                for (int q = 0; q < EPT; ++q) h[q] = cfma(w, A[it.item(q) + off], h[q]);
              }
            }
    #pragma unroll
            for (int q = 0; q < EPT; ++q) {
              const C x = chi[it.item(q)];
              s += x.x * h[q].y - x.y * h[q].x;       // Im(conj(chi) * h)
            }
          }
        } else {
    #pragma unroll
          for (int q = 0; q < EPT; ++q) {
            if (!it.ok(q)) continue;
            const int xi = (it.dig(q) >> (4 * node)) & 15;
            const int base = (t * g.n_loc + xi) * g.SH;
            C h = mkc((R)0, (R)0);
            for (int e = 0; e < g.SH; ++e) {
              const C w = hv[base + e];
              if (w.x != (R)0 || w.y != (R)0) h = cfma(w, A[it.item(q) + sm.hc_off[base + e]], h);
            }
            const C x = chi[it.item(q)];
            s += x.x * h.y - x.y * h.x;       // Im(conj(chi) * h)
          }
        }
        const int ct = g.cterm_ctrl[t];
    #pragma unroll
        for (int c = 0; c < KT_MAX_CTRL; ++c)
          if (c == ct) sc[c] += s;
      }
      // FP64 block reduction of the per-control sums: four slots when there are at most four controls
      // (FP64 runs at 1/64 of the FP32 rate here, and every slot costs additions in each lane)
      int vstride = KT_MAX_CTRL;
      if (g.n_ctrl <= 4) {
        double v[4];
    #pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = c < g.n_ctrl ? (double)sc[c] : 0.0;
        reduce_tau<4>(v, g, sm.red, sm.tsc + TS_V0 * g.T);
        vstride = 4;
      } else {
        double v[KT_MAX_CTRL];
    #pragma unroll
        for (int c = 0; c < KT_MAX_CTRL; ++c) v[c] = c < g.n_ctrl ? (double)sc[c] : 0.0;
        reduce_tau<KT_MAX_CTRL>(v, g, sm.red, sm.tsc + TS_V0 * g.T);
      }
      if (threadIdx.x < g.n_ctrl) {
        double s = 0.0;
        for (int t = 0; t < g.T; ++t) s += sm.tsc[TS_V0 * g.T + t * vstride + threadIdx.x];
        // a sweep keeps two sets of partials (interval parity): a CTA may write the next interval's
        // while a slower one still reads this interval's
        a.partials[(sweep ? (size_t)(j & 1) * g.n_tiles * g.n_ctrl : 0) + (size_t)tile * g.n_ctrl + threadIdx.x] = s;
      }
      store_pending = store_pending || stored;
      end_fwd_tile(sm, persist);
      // every thread is done with this tile's chi (the barrier above): the third buffer takes the next tile's
      if (persist && need_chi && g.prefetch_chi && next < g.n_tiles && threadIdx.x == 0)
        bulk_load(sm.bufC, (const C *)a.chi_t + (size_t)next * g.tile_elems, tile_bytes, &sm.mbar[1]);
    }   // tiles of this CTA
    // Delta eps of interval j+1 from the partials of all tiles: every thread adds a fixed, contiguous
    // chunk of the tiles and a fixed shuffle/warp tree adds the chunks -- the same order on every run
    // for a given tile count and block size.  The new pulse value goes to sm.eps (the next interval of
    // a sweep) and, with write_out, to deps / eps_new.
    auto finish_update = [&](const double *part, bool write_out) {
      const int chunk = (g.n_tiles + (int)blockDim.x - 1) / (int)blockDim.x;
      const int t0 = threadIdx.x * chunk, t1 = min(g.n_tiles, t0 + chunk);
      for (int c = 0; c < g.n_ctrl; ++c) {
        double v = 0.0;
        for (int t = t0; t < t1; ++t) v += __ldcg(part + (size_t)t * g.n_ctrl + c);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sm.red[(threadIdx.x >> 5) * 8 + c] = v;
      }
      __syncthreads();
      if (threadIdx.x < g.n_ctrl) {
        const int c = threadIdx.x;
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm.red[w * 8 + c];
        const size_t idx = (size_t)c * a.nt + j;   // interval j+1 (0-based index j)
        const double de = (sweep ? fin_scale : a.shape[idx] / (g.lam[c] * g.M_norm)) * s;
        const double en = (sweep ? fin_eold : a.eps_old[idx]) + de;
        if (write_out) {
          a.deps[idx] = de;
          a.eps_new[idx] = en;
          if (!isfinite(de)) set_status(a.status, KT_DEV_NONFINITE);
          if (fabs(en) > g.eps_bound) set_status(a.status, KT_DEV_RANGE);
        }
        sm.eps[c] = en;
      }
    };
    if (sweep) {
      if (j == a.nt) break;
      if (!need_chi) continue;                 // guess sweep: nothing to exchange between intervals
      if (!grid_barrier(a.sync, sync_gen, &sm.flag[6], a.status)) break;   // timed out: results void
      ++sync_gen;
      finish_update(a.partials + (size_t)(j & 1) * g.n_tiles * g.n_ctrl, blockIdx.x == 0);
      continue;
    }
    if (!a.overlap || j == a.nt || !a.finish) {   // no update sum here (a shard sums after its exchange)
      if (threadIdx.x == 0 && store_pending) bulk_store_wait();
      return;
    }
    // ---------------- last CTA: Delta eps of interval j+1, summed in tile order ----------------
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned ticket = atomicAdd(a.counter, 1u);
      sm.flag[3] = (ticket == (unsigned)(gridDim.x - 1));
    }
    __syncthreads();
    if (threadIdx.x == 0 && store_pending) bulk_store_wait();
    if (!sm.flag[3]) return;
    __threadfence();
    finish_update(a.partials, true);
    if (threadIdx.x == 0) *a.counter = 0u;
    return;
  }   // intervals
  if (threadIdx.x == 0 && store_pending) bulk_store_wait();
}

// --------------------------------------------------------------------------------------
// Backward interval kernel: chi(t_{j-1}) = U_j^dag chi(t_j) along each trajectory's record.
// Round rnd propagates piece rnd of the interval (backwards: dt - s_m, s_m - s_{m-1}, ..., s_1)
// and then applies conj(c) L^dag of the jump that bounds it.  One Chebyshev call site.
// With a.forward_replay the same kernel replays a recorded forward pass instead: the image is
// the forward generator's, pieces run forwards (s_1, s_2 - s_1, ..., dt - s_m) and each is
// followed by c L of its jump -- the frozen-record map U_j of the gradient (no bisection).
// Tiles: with g.bwd_grid > 0 the grid holds that many CTAs, each looping over tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...: the tables and the item mapping (which depend on the interval only)
// are built once, and the next tile's input arrives by bulk copy in a third buffer while the current
// tile's series runs (loads alternate between two transaction barriers).  Otherwise one tile per CTA.
// With a.sweep one launch runs the whole backward sweep of its tile, intervals a.j down to 1 (the
// co-states of different trajectories never meet, so the CTAs need no synchronisation): the state
// stays in shared memory from one interval to the next, and each interval's result is stored to its
// co-state slot.
template <typename R, int EPT, int NL, int ACS, bool SWEEP>
__global__ void __launch_bounds__(NL > 0 ? 736 : (sizeof(R) == 8 ? 512 : 1024)) bwd_kernel(KtGeom g, KtGenImage im, KtOps ops, BwdArgs a) {
  typedef typename C2<R>::T C;
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm;
  constexpr bool sweep = SWEEP;   // a.sweep, compiled in
  const bool persist = !sweep && g.bwd_grid > 0;
  carve(g, sizeof(C), smem_raw, &sm, persist);
  const int tau = threadIdx.x % g.T;
  const int j_first = a.j, j_last = sweep ? 1 : a.j;
  if (threadIdx.x < g.n_ctrl) sm.eps[threadIdx.x] = a.eps[threadIdx.x * a.nt + (j_first - 1)];
  if (threadIdx.x < 8) sm.flag[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    mbar_init(&sm.mbar[0], 1);
    mbar_init(&sm.mbar[1], 1);
    mbar_init(&sm.mbar[2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t tile_bytes = (uint32_t)(g.tile_elems * sizeof(C));
  int tile = blockIdx.x;
  if (threadIdx.x == 0)
    bulk_load(sm.bufB, (const C *)a.chi_in + (size_t)tile * g.tile_elems, tile_bytes, &sm.mbar[0]);
  build_tables<R>(g, im, ops, sm, sm.eps, false);
  const bool fw = a.forward_replay != 0;
  Items<EPT, NL> it;
  load_items<EPT, NL>(g, ops, it);
  bool store_pending = false;
  for (int use = 0; tile < g.n_tiles; tile += gridDim.x, ++use) {
    // this tile's input: load number `use`, on barrier use & 1 with phase parity (use >> 1) & 1
    if (!tile_wait(&sm.mbar[use & 1], (use >> 1) & 1, &sm.flag[4], a.status,
                   g.inject_timeout ? &sm.mbar[2] : nullptr)) {
      if (threadIdx.x == 0 && store_pending) bulk_store_wait();
      return;
    }
    const int next = tile + (int)gridDim.x;
    if (persist && next < g.n_tiles && threadIdx.x == 0)   // the third buffer is free: prefetch the next input
      bulk_load(sm.bufC, (const C *)a.chi_in + (size_t)next * g.tile_elems, tile_bytes, &sm.mbar[(use + 1) & 1]);
    for (int j = j_first; j >= j_last; --j) {
      if (j != j_first) {
        // whole sweep: the pulse and the tables of the next interval (every read of the previous
        // interval's tables ended at the barrier after its store)
        if (threadIdx.x < g.n_ctrl) sm.eps[threadIdx.x] = a.eps[threadIdx.x * a.nt + (j - 1)];
        __syncthreads();
        build_tables<R>(g, im, ops, sm, sm.eps, false, true);
      }
      C *chi_out = sweep ? (C *)((char *)a.chi_slots + (size_t)(j - 1) * a.slot_bytes) + (size_t)tile * g.tile_elems
                         : (C *)a.chi_out + (size_t)tile * g.tile_elems;
      if (threadIdx.x == 0) sm.flag[0] = 0;
      if (threadIdx.x == 0 && store_pending) bulk_store_wait();   // A still feeds the previous tile's store
      store_pending = false;
      __syncthreads();
      if (threadIdx.x < g.T) {
        const int t = threadIdx.x, k = tile * g.T + t;
        int nj = 0;
        if (k < g.M) {
          int cur = a.cursor[k];
          if (fw) {
            const int cnt = a.jcount[k];
            while (cur < cnt && a.rec_step[(size_t)k * g.max_jumps + cur] == j && nj < 12) {
              sm.tin[(TI_J0 + nj) * g.T + t] = cur;  // ascending in time
              ++nj;
              ++cur;
            }
            if (cur < cnt && a.rec_step[(size_t)k * g.max_jumps + cur] == j) set_status(a.status, KT_DEV_RECORD_FULL);
          } else {
            while (cur >= 0 && a.rec_step[(size_t)k * g.max_jumps + cur] == j && nj < 12) {
              sm.tin[(TI_J0 + nj) * g.T + t] = cur;  // descending in time
              ++nj;
              --cur;
            }
            if (cur >= 0 && a.rec_step[(size_t)k * g.max_jumps + cur] == j) set_status(a.status, KT_DEV_RECORD_FULL);
          }
          if (a.advance_cursor) a.cursor[k] = cur;
        }
        sm.tin[TI_NJ * g.T + t] = nj;
        atomicMax(&sm.flag[0], nj);
      }
      __syncthreads();
      C *A = (C *)sm.bufA;
      C *B = (C *)sm.bufB;
      const int rounds = sm.flag[0];
      C acc[EPT];
      for (int rnd = 0; rnd <= rounds; ++rnd) {
        if (rounds == 0) {
          uniform_coefs<R>(g, sm, im.cheb_full);
        } else if (threadIdx.x < g.T) {
          const int t = threadIdx.x, k = tile * g.T + t, nj = sm.tin[TI_NJ * g.T + t];
          double len = 0.0;
          if (rnd <= nj) {
            const double *rs = a.rec_s + (size_t)k * g.max_jumps;
            if (fw) {   // pieces forwards: s_1 - 0, s_2 - s_1, ..., dt - s_m
              const double lo = (rnd == 0) ? 0.0 : rs[sm.tin[(TI_J0 + rnd - 1) * g.T + t]];
              const double hi = (rnd < nj) ? rs[sm.tin[(TI_J0 + rnd) * g.T + t]] : g.dt;
              len = hi - lo;
            } else {    // pieces backwards: dt - s_m, s_m - s_{m-1}, ..., s_1 - 0
              const double hi = (rnd == 0) ? g.dt : rs[sm.tin[(TI_J0 + rnd - 1) * g.T + t]];
              const double lo = (rnd < nj) ? rs[sm.tin[(TI_J0 + rnd) * g.T + t]] : 0.0;
              len = hi - lo;
            }
          }
          tau_coefs<R>(g, sm, t, fw ? g.c_fwd : g.c_bwd, len);
        }
        // B holds the vector to propagate
  #pragma unroll
        for (int q = 0; q < EPT; ++q)
          if (it.ok(q)) A[it.item(q)] = B[it.item(q)];
        __syncthreads();
        // FP32: the other nodes' rows in registers (measured 2 % faster); FP64 has no registers to spare
        cheb_dispatch<R, EPT, NL, ACS, sizeof(R) == 4>(g, im, sm, it, g.K, acc);
        if (rnd == rounds) break;
  #pragma unroll
        for (int q = 0; q < EPT; ++q)
          if (it.ok(q)) A[it.item(q)] = acc[q];
        __syncthreads();
        const int nj = sm.tin[TI_NJ * g.T + tau];
        const int k = tile * g.T + tau;
  #pragma unroll
        for (int q = 0; q < EPT; ++q) {
          if (!it.ok(q)) continue;
          C y = A[it.item(q)];
          if (rnd < nj) {
            const size_t ri = (size_t)k * g.max_jumps + sm.tin[(TI_J0 + rnd) * g.T + tau];
            const C z = lind_item<R>(g, ops, a.rec_ch[ri], fw ? 0 : 1, A, it.item(q), it.dig(q));
            const R cn = (R)a.rec_c[ri];
            y = mkc(cn * z.x, cn * z.y);
          }
          B[it.item(q)] = y;
        }
        __syncthreads();
      }
      // chi(t_{j-1}) of the whole tile: into A, then one bulk store (completed before A is reused)
  #pragma unroll
      for (int q = 0; q < EPT; ++q)
        if (it.ok(q)) A[it.item(q)] = acc[q];
      if (sweep && j > j_last) {
        // the next interval starts from this result (B's last reads ended at the rounds' barrier)
  #pragma unroll
        for (int q = 0; q < EPT; ++q)
          if (it.ok(q)) B[it.item(q)] = acc[q];
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (threadIdx.x == 0) bulk_store(chi_out, A, tile_bytes);
      store_pending = true;
    }   // intervals
    // the prefetched input becomes this CTA's input buffer; the old one (free) the next prefetch target
    void *tmp = sm.bufB;
    sm.bufB = sm.bufC;
    sm.bufC = tmp;
  }
  if (threadIdx.x == 0 && store_pending) bulk_store_wait();
}

}  // namespace kt
