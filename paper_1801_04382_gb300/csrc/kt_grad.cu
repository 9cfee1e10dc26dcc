// Gradient of the trajectory functional with respect to the piecewise-constant controls, with
// the jump record of the forward pass held fixed (the differentiable object defined by freezing
// (interval, s*, channel, c) of every jump; J_T is invariant to the c's).
//
//   dJ_T/deps_ij = -(2/M) sum_k Re <chi~_k(t_j)| dU_kj/deps_i |psi_k(t_{j-1})>,
//
// U_kj = P(tau_m) c_m L ... c_1 L P(tau_0) the trajectory's map over interval j (pieces between its
// recorded jumps), chi~ the co-state of the exact boundary propagated backwards along the same
// record.  By the product rule the bracket is a sum over pieces q of <W_q| dP(tau_q) |Z_q>, Z_q the
// state at the start of piece q and W_q the co-state at its end.  dP(tau)/deps_i is evaluated
// exactly with the Chebyshev series of the block-triangular generator [[G, H_i], [0, G]] applied
// to [0; Z]: T_k of that block matrix carries dT_k(Ghat)/deps in its upper-right block, so the
// recurrences z_{k+1} = 2 Ghat z_k - z_{k-1} and y_{k+1} = 2 (Ghat y_k + Hhat_i z_k) - y_{k-1}
// (y_0 = 0, y_1 = Hhat_i z_0) give dP/deps_i Z = sum_k a_k y_k with the propagator's own
// coefficients a_k (the same constants c, r: only Ghat depends on eps).
//
// One CTA per trajectory, gathered from the problem's interleaved tile layout.
#include "kt_device.cuh"

namespace kt {

__host__ __device__ inline size_t grad_carve(const KtGeom &g1, int esz, char *base, Smem *s, void **D) {
  size_t off = carve(g1, esz, base, s, true);
  off = align_up(off, 16);
  if (D) *D = base ? base + off : nullptr;
  off += (size_t)g1.tile_elems * esz;
  return align_up(off, 16);
}

// trajectory k of a tile-layout array (T_layout interleaved) -> dst[x]
template <typename R, int EPT, class IT>
__device__ __forceinline__ void gather_traj(const IT &it, const typename C2<R>::T *tiles, int k, int T_layout,
                                            int tel, typename C2<R>::T *dst) {
  const typename C2<R>::T *src = tiles + (size_t)(k / T_layout) * tel + (k % T_layout);
#pragma unroll
  for (int q = 0; q < EPT; ++q)
    if (it.ok(q)) dst[it.item(q)] = src[(size_t)it.item(q) * T_layout];
}

// (H_c / r) v at one item (control factor c, scaled like the generator)
template <typename R>
__device__ __forceinline__ typename C2<R>::T hc_item(const KtGeom &g, const Smem &sm, int c,
                                                     const typename C2<R>::T *v, int item, uint32_t dig, R invr) {
  typedef typename C2<R>::T C;
  const C *hv = (const C *)sm.hc_val;
  const int xi = (dig >> (4 * g.ctrl_node[c])) & 15;
  const int base = (c * g.n_loc + xi) * g.SH;
  C h = mkc((R)0, (R)0);
  for (int e = 0; e < g.SH; ++e) {
    const C w = hv[base + e];
    if (w.x != (R)0 || w.y != (R)0) h = cfma(w, v[item + sm.hc_off[base + e]], h);
  }
  return mkc(h.x * invr, h.y * invr);
}

// acc = sum_k a_k y_k, the derivative along control c of sum_k a_k T_k(Ghat) z0 (z0 in A, synced).
// Uses A, B (z recurrence) and C, D (y recurrence).  Ends synchronised.
template <typename R, int EPT, class IT>
__device__ void aug_run(const KtGeom &g, const KtGenImage &im, const Smem &sm, const IT &it, int K, int c,
                        typename C2<R>::T *Dbuf, typename C2<R>::T (&acc)[EPT]) {
  typedef typename C2<R>::T C;
  C *A = (C *)sm.bufA, *B = (C *)sm.bufB, *Cb = (C *)sm.bufC, *D = Dbuf;
  const C *cf = (const C *)sm.coef;
  const R invr = (R)(1.0 / g.r);
  C dv[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    dv[q] = it.ok(q) ? diag_of<R>(g, sm, it.dig(q)) : mkc((R)0, (R)0);
    acc[q] = mkc((R)0, (R)0);
    if (it.ok(q)) Cb[it.item(q)] = mkc((R)0, (R)0);   // y_0 = 0
  }
  if (K < 2) { __syncthreads(); return; }
  const C c1 = cf[1];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    if (!it.ok(q)) continue;
    const int i = it.item(q);
    B[i] = apply_item<R>(g, im, sm, A, i, it.dig(q), dv[q]);       // z_1 = Ghat z_0
    const C y1 = hc_item<R>(g, sm, c, A, i, it.dig(q), invr);       // y_1 = Hhat z_0
    D[i] = y1;
    acc[q] = cfma(c1, y1, acc[q]);
  }
  __syncthreads();
  C *Pz = A, *Qz = B, *Py = Cb, *Qy = D;
  for (int k = 2; k < K; ++k) {
    const C ak = cf[k];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      if (!it.ok(q)) continue;
      const int i = it.item(q);
      const C tz = apply_item<R>(g, im, sm, Qz, i, it.dig(q), dv[q]);
      C ty = apply_item<R>(g, im, sm, Qy, i, it.dig(q), dv[q]);
      const C hz = hc_item<R>(g, sm, c, Qz, i, it.dig(q), invr);
      ty.x += hz.x;
      ty.y += hz.y;
      const C oz = Pz[i], oy = Py[i];
      const C nz = mkc(tz.x + tz.x - oz.x, tz.y + tz.y - oz.y);
      const C ny = mkc(ty.x + ty.x - oy.x, ty.y + ty.y - oy.y);
      Pz[i] = nz;
      Py[i] = ny;
      acc[q] = cfma(ak, ny, acc[q]);
    }
    __syncthreads();
    C *t1 = Pz; Pz = Qz; Qz = t1;
    C *t2 = Py; Py = Qy; Qy = t2;
  }
}

// Fiber form of (H_c / r) v for the thread's fiber (tile width 1): a control on the last node
// takes row q of its factor for element q, a control on another node one row for the whole fiber.
// Same entries and order as hc_item.
template <typename R, int NL>
__device__ __forceinline__ void hc_fiber(const KtGeom &g, const Smem &sm, int c, const typename C2<R>::T *v, int base,
                                         uint32_t fdig, R invr, typename C2<R>::T (&h)[NL]) {
  typedef typename C2<R>::T C;
  const C *hv = (const C *)sm.hc_val;
  const int node = g.ctrl_node[c];
#pragma unroll
  for (int q = 0; q < NL; ++q) h[q] = mkc((R)0, (R)0);
  if (node == g.n_nodes - 1) {
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      const int b = (c * g.n_loc + q) * g.SH;
      for (int e = 0; e < g.SH; ++e) {
        const C w = hv[b + e];
        if (w.x != (R)0 || w.y != (R)0) h[q] = cfma(w, v[base + q + sm.hc_off[b + e]], h[q]);
      }
    }
  } else {
    const int b = (c * g.n_loc + ((fdig >> (4 * node)) & 15)) * g.SH;
    for (int e = 0; e < g.SH; ++e) {
      const C w = hv[b + e];
      if (w.x != (R)0 || w.y != (R)0) {
        const int off = sm.hc_off[b + e];
#pragma unroll
        for (int q = 0; q < NL; ++q) h[q] = cfma(w, v[base + off + q], h[q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NL; ++q) h[q] = mkc(h[q].x * invr, h[q].y * invr);
}

// aug_run in the fiber mapping with tile width 1, for the cavity structure with real / imaginary
// coupling classes: the same two recurrences, Ghat applied by apply_acs.
template <typename R, int NC, class IT>
__device__ void aug_run_acs(const KtGeom &g, const KtGenImage &im, const Smem &sm, const IT &it, int K, int c,
                            typename C2<R>::T *Dbuf, typename C2<R>::T (&acc)[3 * (NC + 1)]) {
  typedef typename C2<R>::T C;
  constexpr int NL = 3 * (NC + 1);
  C *A = (C *)sm.bufA, *B = (C *)sm.bufB, *Cb = (C *)sm.bufC, *D = Dbuf;
  const C *cf = (const C *)sm.coef;
  const C *dg = (const C *)sm.diag;
  const R invr = (R)(1.0 / g.r);
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
#pragma unroll
  for (int q = 0; q < NL; ++q) {
    acc[q] = mkc((R)0, (R)0);
    if (ok) Cb[base + q] = mkc((R)0, (R)0);   // y_0 = 0
  }
  if (K < 2) { __syncthreads(); return; }
  C v[NL], t[NL], h[NL];
  RowCache<R> rc;
  if (ok) load_rows<R, NL>(g, sm, fdig, rc);
  if (ok) {
#pragma unroll
    for (int q = 0; q < NL; ++q) v[q] = A[base + q];
    apply_acs<R, NC, 1, true, true>(g, im, sm, A, base, fdig, Df, v, t, rc);      // z_1 = Ghat z_0
    hc_fiber<R, NL>(g, sm, c, A, base, fdig, invr, h);                // y_1 = Hhat z_0
    const C c1 = cf[1];
#pragma unroll
    for (int q = 0; q < NL; ++q) {
      B[base + q] = t[q];
      D[base + q] = h[q];
      acc[q] = cfma(c1, h[q], acc[q]);
    }
  }
  __syncthreads();
  C *Pz = A, *Qz = B, *Py = Cb, *Qy = D;
  for (int k = 2; k < K; ++k) {
    if (ok) {
      const C ak = cf[k];
#pragma unroll
      for (int q = 0; q < NL; ++q) v[q] = Qz[base + q];
      apply_acs<R, NC, 1, true, true>(g, im, sm, Qz, base, fdig, Df, v, t, rc);
      hc_fiber<R, NL>(g, sm, c, Qz, base, fdig, invr, h);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const C oz = Pz[base + q];
        Pz[base + q] = mkc(t[q].x + t[q].x - oz.x, t[q].y + t[q].y - oz.y);
        v[q] = Qy[base + q];
      }
      apply_acs<R, NC, 1, true, true>(g, im, sm, Qy, base, fdig, Df, v, t, rc);
#pragma unroll
      for (int q = 0; q < NL; ++q) {
        const C ty = mkc(t[q].x + h[q].x, t[q].y + h[q].y);
        const C oy = Py[base + q];
        const C ny = mkc(ty.x + ty.x - oy.x, ty.y + ty.y - oy.y);
        Py[base + q] = ny;
        acc[q] = cfma(ak, ny, acc[q]);
      }
    }
    __syncthreads();
    C *t1 = Pz; Pz = Qz; Qz = t1;
    C *t2 = Py; Py = Qy; Qy = t2;
  }
}

// NL = 0: strided items (EPT per thread); NL = 9 with ACS = 4: fiber mapping, tile width 1,
// cavity structure with real / imaginary coupling classes.
template <typename R, int EPT, int NL, int ACS>
__global__ void __launch_bounds__(NL > 0 ? 96 : (EPT == 4 ? 256 : 1024), NL > 0 ? 5 : 1)
    grad_kernel(KtGeom g, int T_layout, int tel, KtGenImage imf, KtGenImage imb, KtOps ops, GradArgs a) {
  typedef typename C2<R>::T C;
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm;
  void *Dv = nullptr;
  grad_carve(g, sizeof(C), smem_raw, &sm, &Dv);
  C *D = (C *)Dv;
  C *A = (C *)sm.bufA, *B = (C *)sm.bufB;
  const int k = blockIdx.x;
  const int j = a.j;
  const size_t rb = (size_t)k * g.max_jumps;
  if (threadIdx.x < g.n_ctrl) sm.eps[threadIdx.x] = a.eps[threadIdx.x * a.nt + (j - 1)];
  if (threadIdx.x < 8) sm.flag[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    // records of interval j in ascending time: walk down from the backward cursor, then reverse
    int cur = a.cursor[k], n = 0, idx[12];
    while (cur >= 0 && a.rec_step[rb + cur] == j && n < 12) idx[n++] = cur--;
    if (cur >= 0 && a.rec_step[rb + cur] == j) set_status(a.status, KT_DEV_RECORD_FULL);
    for (int m = 0; m < n; ++m) sm.tin[TI_J0 + m] = idx[n - 1 - m];
    sm.tin[TI_NJ] = n;
  }
  __syncthreads();
  const int m = sm.tin[TI_NJ];
  Items<EPT, NL> it;
  load_items<EPT, NL>(g, ops, it);
  const C *psi_t = (const C *)a.psi_prev;
  const C *chi_t = (const C *)a.chi_t;
  // piece boundaries s_0 = 0 < s_1 < ... < s_m < s_{m+1} = dt
  auto sb = [&](int p) -> double { return p == 0 ? 0.0 : (p > m ? g.dt : a.rec_s[rb + sm.tin[TI_J0 + p - 1]]); };
  double part[KT_MAX_CTRL];
  for (int c = 0; c < KT_MAX_CTRL; ++c) part[c] = 0.0;
  C acc[EPT], wq[EPT], zq[EPT];
  for (int q = 0; q <= m; ++q) {
    // phase 0: W_q = chi~ taken back over pieces m..q+1 (adjoint generator, jumps c L^dag);
    // phase 1: Z_q = psi(t_{j-1}) taken forward over pieces 0..q-1 (jumps c L)
    for (int ph = 0; ph < 2; ++ph) {
      const bool adj = ph == 0;
      const KtGenImage &imd = adj ? imb : imf;
      const int np = adj ? m - q : q;
      gather_traj<R, EPT>(it, adj ? chi_t : psi_t, k, T_layout, tel, A);
      if (np > 0 || !adj) build_tables<R>(g, imd, ops, sm, sm.eps, !adj);
      __syncthreads();
      for (int step = 0; step < np; ++step) {
        const int p = adj ? m - step : step;
        if (threadIdx.x == 0) tau_coefs<R>(g, sm, 0, adj ? g.c_bwd : g.c_fwd, sb(p + 1) - sb(p));
        __syncthreads();
        cheb_run<R, EPT>(g, imd, sm, it, g.K, acc);
#pragma unroll
        for (int qq = 0; qq < EPT; ++qq)
          if (it.ok(qq)) A[it.item(qq)] = acc[qq];
        __syncthreads();
        const size_t ri = rb + sm.tin[TI_J0 + (adj ? p - 1 : p)];
        const R cn = (R)a.rec_c[ri];
#pragma unroll
        for (int qq = 0; qq < EPT; ++qq)
          if (it.ok(qq)) {
            const C z = lind_item<R>(g, ops, a.rec_ch[ri], adj ? 1 : 0, A, it.item(qq), it.dig(qq));
            B[it.item(qq)] = mkc(cn * z.x, cn * z.y);
          }
        __syncthreads();
#pragma unroll
        for (int qq = 0; qq < EPT; ++qq)
          if (it.ok(qq)) A[it.item(qq)] = B[it.item(qq)];
        __syncthreads();
      }
#pragma unroll
      for (int qq = 0; qq < EPT; ++qq) {
        const C v = it.ok(qq) ? A[it.item(qq)] : mkc((R)0, (R)0);
        if (adj) wq[qq] = v;
        else zq[qq] = v;
      }
      __syncthreads();
    }
    // ---- derivative of piece q along every control: <W_q| dP(tau_q)/deps_c |Z_q>
    if (threadIdx.x == 0) {
      if (m == 0) {
        for (int e = 0; e < g.K; ++e) ((C *)sm.coef)[e] = from_kc<C>(imf.cheb_full[e]);
      } else {
        tau_coefs<R>(g, sm, 0, g.c_fwd, sb(q + 1) - sb(q));
      }
    }
    for (int c = 0; c < g.n_ctrl; ++c) {
#pragma unroll
      for (int qq = 0; qq < EPT; ++qq)
        if (it.ok(qq)) A[it.item(qq)] = zq[qq];
      __syncthreads();
      if constexpr (ACS == 4) aug_run_acs<R, NL / 3 - 1>(g, imf, sm, it, g.K, c, D, acc);
      else aug_run<R, EPT>(g, imf, sm, it, g.K, c, D, acc);
      double sacc = 0.0;
#pragma unroll
      for (int qq = 0; qq < EPT; ++qq)
        if (it.ok(qq)) sacc += (double)(wq[qq].x * acc[qq].x + wq[qq].y * acc[qq].y);   // Re(conj(W) y)
      part[c] += sacc;
    }
  }
  reduce_tau<KT_MAX_CTRL>(part, g, sm.red, sm.tsc + TS_V0 * g.T);
  if (threadIdx.x < g.n_ctrl) a.partials[(size_t)k * g.n_ctrl + threadIdx.x] = sm.tsc[TS_V0 * g.T + threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(a.counter, 1u);
    sm.flag[3] = (ticket == (unsigned)(gridDim.x - 1));
  }
  __syncthreads();
  if (!sm.flag[3]) return;
  __threadfence();
  const int chunk = ((int)gridDim.x + blockDim.x - 1) / blockDim.x;
  const int t0 = threadIdx.x * chunk, t1 = min((int)gridDim.x, t0 + chunk);
  for (int c = 0; c < g.n_ctrl; ++c) {
    double v = 0.0;
    for (int t = t0; t < t1; ++t) v += __ldcg(a.partials + (size_t)t * g.n_ctrl + c);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm.red[(threadIdx.x >> 5) * 8 + c] = v;
  }
  __syncthreads();
  if (threadIdx.x < g.n_ctrl) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sm.red[w * 8 + threadIdx.x];
    const double gr = -2.0 / (double)g.M * s;
    a.grad[(size_t)threadIdx.x * a.nt + (j - 1)] = gr;
    if (!isfinite(gr)) set_status(a.status, KT_DEV_NONFINITE);
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <typename R, int EPT, int NL, int ACS>
static cudaError_t launch_grad_t(const KtGeom &g1, int T_layout, int tel, const KtGenImage &imf,
                                 const KtGenImage &imb, const KtOps &ops, const GradArgs &a, cudaStream_t st) {
  const cudaError_t attr = kt_allow_large_smem((const void *)grad_kernel<R, EPT, NL, ACS>);
  if (attr != cudaSuccess) return attr;
  const size_t smem = grad_carve(g1, sizeof(typename C2<R>::T), nullptr, nullptr, nullptr);
  grad_kernel<R, EPT, NL, ACS><<<g1.M, g1.nthreads, smem, st>>>(g1, T_layout, tel, imf, imb, ops, a);
  return cudaGetLastError();
}

}  // namespace kt

size_t kt_grad_smem_bytes(const KtGeom &g1, int elem_bytes) {
  return kt::grad_carve(g1, elem_bytes, nullptr, nullptr, nullptr);
}

cudaError_t kt_launch_grad(int fp64, int ept, const KtGeom &g1, int T_layout, int tel, const KtGenImage &imf,
                           const KtGenImage &imb, const KtOps &ops, const GradArgs &a, cudaStream_t st) {
  if (fp64) {
    switch (ept) {
      case 4: return kt::launch_grad_t<double, 4, 0, 0>(g1, T_layout, tel, imf, imb, ops, a, st);
      case 8: return kt::launch_grad_t<double, 8, 0, 0>(g1, T_layout, tel, imf, imb, ops, a, st);
      case -409: return kt::launch_grad_t<double, 9, 9, 4>(g1, T_layout, tel, imf, imb, ops, a, st);
    }
  } else {
    switch (ept) {
      case 4: return kt::launch_grad_t<float, 4, 0, 0>(g1, T_layout, tel, imf, imb, ops, a, st);
      case 8: return kt::launch_grad_t<float, 8, 0, 0>(g1, T_layout, tel, imf, imb, ops, a, st);
      case -409: return kt::launch_grad_t<float, 9, 9, 4>(g1, T_layout, tel, imf, imb, ops, a, st);
    }
  }
  return cudaErrorInvalidValue;
}
