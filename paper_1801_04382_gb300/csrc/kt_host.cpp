// Host runtime of the trajectory-parallel Krotov library: validation, assembly of the
// structured MCWF generator (a1), Chebyshev set-up (a2), device memory, and the sweep
// schedulers behind the C ABI declared in include/krotov_traj.h.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/krotov_traj.h"
#include "kt_common.h"
#include "kt_kernels.h"

typedef std::complex<double> cd;

namespace {

thread_local std::string g_err;

kt_status fail(kt_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define KT_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(KT_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// ---------------------------------------------------------------------------- NCCL, loaded at run time
// The library does not link NCCL: a sharded problem loads it with dlopen (the caller may name the
// file) and uses four entry points of its C API.
struct NcclApi {
  typedef int (*GetUniqueId)(void *id);
  typedef int (*CommInitRank)(void **comm, int nranks, std::array<char, 128> id, int rank);
  typedef int (*AllGather)(const void *send, void *recv, size_t count, int dtype, void *comm, cudaStream_t st);
  typedef int (*CommDestroy)(void *comm);
  typedef const char *(*ErrorString)(int r);
  void *handle = nullptr;
  GetUniqueId get_unique_id = nullptr;
  CommInitRank comm_init_rank = nullptr;
  AllGather all_gather = nullptr;
  CommDestroy comm_destroy = nullptr;
  ErrorString error_string = nullptr;
};
const int kNcclDouble = 8;   // ncclFloat64

NcclApi g_nccl;
std::mutex g_nccl_mu;

kt_status nccl_load(const char *path) {
  std::lock_guard<std::mutex> lock(g_nccl_mu);
  if (g_nccl.handle) return KT_OK;
  void *h = dlopen(path && *path ? path : "libnccl.so.2", RTLD_NOW | RTLD_GLOBAL);
  if (!h) return fail(KT_ERR_UNSUPPORTED, "NCCL not found (%s)", dlerror());
  NcclApi api;
  api.handle = h;
  api.get_unique_id = (NcclApi::GetUniqueId)dlsym(h, "ncclGetUniqueId");
  api.comm_init_rank = (NcclApi::CommInitRank)dlsym(h, "ncclCommInitRank");
  api.all_gather = (NcclApi::AllGather)dlsym(h, "ncclAllGather");
  api.comm_destroy = (NcclApi::CommDestroy)dlsym(h, "ncclCommDestroy");
  api.error_string = (NcclApi::ErrorString)dlsym(h, "ncclGetErrorString");
  if (!api.get_unique_id || !api.comm_init_rank || !api.all_gather || !api.comm_destroy || !api.error_string) {
    dlclose(h);
    return fail(KT_ERR_UNSUPPORTED, "the NCCL library lacks an entry point this library uses");
  }
  g_nccl = api;
  return KT_OK;
}

// ---------------------------------------------------------------------------- structured generator
// Pair hop between two different nodes: kind 0 coef a_dst^dag a_src (the cascade, L^dag L cross
// terms), kind 1 coef a_dst a_src and kind 2 coef a_dst^dag a_src^dag (the L rho L^dag term of a
// density matrix in Liouville space, and its adjoint).
struct Pair {
  int dst, src;
  cd coef;
  int kind = 0;
};

// Structured generator: node factors, control terms and pair hops.  A control term is one factor
// of a control on one node (ctrl_node[t], control term_ctrl[t]); an ordinary model has one term
// per control, the Liouville-space generator of a density matrix two (the ket and the bra node).
struct Gen {
  int N = 0, nl = 0, n_ctrl = 0;
  std::vector<cd> loc;    // [N][nl][nl]
  std::vector<cd> ctrl;   // [n_terms][nl][nl] (per unit eps)
  std::vector<int> ctrl_node;   // [n_terms] node of each term
  std::vector<int> term_ctrl;   // [n_terms] control of each term
  std::vector<Pair> pairs;
};

inline cd at(const std::vector<cd> &m, int base, int nl, int x, int y) { return m[base + x * nl + y]; }

// a^dag a of the ladder factor
std::vector<cd> adag_a(const std::vector<cd> &a, int nl) {
  std::vector<cd> out(nl * nl);
  for (int x = 0; x < nl; ++x)
    for (int y = 0; y < nl; ++y) {
      cd s = 0;
      for (int z = 0; z < nl; ++z) s += std::conj(a[z * nl + x]) * a[z * nl + y];
      out[x * nl + y] = s;
    }
  return out;
}

// Adjoint-direction generator -G^dag (co-state propagation: exp(+i H_eff^dag s) = exp(-i (-H_eff^dag) s)).
Gen minus_adjoint(const Gen &f) {
  Gen b = f;
  const int nl = f.nl;
  for (size_t base = 0; base < f.loc.size(); base += nl * nl)
    for (int x = 0; x < nl; ++x)
      for (int y = 0; y < nl; ++y) b.loc[base + x * nl + y] = -std::conj(f.loc[base + y * nl + x]);
  for (size_t base = 0; base < f.ctrl.size(); base += nl * nl)
    for (int x = 0; x < nl; ++x)
      for (int y = 0; y < nl; ++y) b.ctrl[base + x * nl + y] = -std::conj(f.ctrl[base + y * nl + x]);
  // (c a_d^dag a_s)^dag = conj(c) a_s^dag a_d; (c a_d a_s)^dag = conj(c) a_d^dag a_s^dag and back
  for (size_t p = 0; p < f.pairs.size(); ++p) {
    const Pair &q = f.pairs[p];
    if (q.kind == 0) b.pairs[p] = Pair{q.src, q.dst, -std::conj(q.coef), 0};
    else b.pairs[p] = Pair{q.dst, q.src, -std::conj(q.coef), q.kind == 1 ? 2 : 1};
  }
  return b;
}

struct Bounds {
  double lo, hi, damp;
};

// Spectral bounds of a direction's generator: real parts in [lo, hi] from Gershgorin discs of
// each node's Hermitian part (the node terms act on different factors, so their spectra add),
// plus the norms of the pair terms; |imaginary parts| <= damp likewise for the anti-Hermitian part.
Bounds gen_bounds(const Gen &g, double amax, double E) {
  const int nl = g.nl;
  Bounds b{0.0, 0.0, 0.0};
  for (int i = 0; i < g.N; ++i) {
    double lo = 1e300, hi = -1e300, dmax = 0.0;
    for (int x = 0; x < nl; ++x) {
      auto herm = [&](const std::vector<cd> &m, int base, int y) {
        return 0.5 * (m[base + x * nl + y] + std::conj(m[base + y * nl + x]));
      };
      auto anti = [&](const std::vector<cd> &m, int base, int y) {
        return (m[base + x * nl + y] - std::conj(m[base + y * nl + x])) / cd(0.0, 2.0);
      };
      const int lb = i * nl * nl;
      double cen = herm(g.loc, lb, x).real(), rad = 0.0;
      double acen = std::abs(anti(g.loc, lb, x)), arad = 0.0;
      for (size_t c = 0; c < g.ctrl_node.size(); ++c)
        if (g.ctrl_node[c] == i) {
          rad += E * std::abs(herm(g.ctrl, c * nl * nl, x).real());
          arad += E * std::abs(anti(g.ctrl, c * nl * nl, x));
        }
      for (int y = 0; y < nl; ++y) {
        if (y == x) continue;
        rad += std::abs(herm(g.loc, lb, y));
        arad += std::abs(anti(g.loc, lb, y));
        for (size_t c = 0; c < g.ctrl_node.size(); ++c)
          if (g.ctrl_node[c] == i) {
            rad += E * std::abs(herm(g.ctrl, c * nl * nl, y));
            arad += E * std::abs(anti(g.ctrl, c * nl * nl, y));
          }
      }
      lo = std::min(lo, cen - rad);
      hi = std::max(hi, cen + rad);
      dmax = std::max(dmax, acen + arad);
    }
    b.lo += lo;
    b.hi += hi;
    b.damp += dmax;
  }
  for (const Pair &p : g.pairs) {
    const double nrm = std::abs(p.coef) * amax * amax;
    b.lo -= nrm;
    b.hi += nrm;
    b.damp += nrm;
  }
  return b;
}

// Field-of-values bounds of the forward generator G(eps) = G0 + sum_c eps_c dG/deps_c for all
// |eps_c| <= E, from Gershgorin discs of whole rows of the full-space operator: the real parts of
// W(G) are those of W((G + G^dag)/2) and the imaginary parts those of W((G - G^dag)/(2i)), each
// inside the union of its row discs (centre the diagonal entry at the worst eps, radius the
// off-diagonal row sum with every control at |eps_c| = E).  Whole rows are tighter than the sum of
// per-node bounds (a row never meets the worst case of every node at once).  The backward
// generator -G^dag has Hermitian part -Herm(G) and the same anti-Hermitian part, so its bounds
// follow.  Entries are enumerated with the kernels' own indexing (digits, node strides, pair hops).
Bounds row_bounds(const Gen &g, const std::vector<int> &lo_dl, const std::vector<cd> &lo_val,
                  const std::vector<int> &ra_dl, const std::vector<cd> &ra_val, int d, const int *stride, double E) {
  const int nl = g.nl, N = g.N, nc = g.n_ctrl, nterm = (int)g.ctrl_node.size();
  // entries of G0 (m = 0) and of dG/deps_c (m = 1 + c), keyed by row * d + column
  std::vector<std::unordered_map<long long, cd>> mats(1 + nc);
  auto add = [&](int m, long long x, long long y, cd v) {
    if (v != 0.0) mats[m][x * d + y] += v;
  };
  for (int x = 0; x < d; ++x) {
    int dig[KT_MAX_NODES];
    for (int i = 0; i < N; ++i) dig[i] = (x / stride[i]) % nl;
    for (int i = 0; i < N; ++i)
      for (int y = 0; y < nl; ++y) {
        const long long col = x + (long long)(y - dig[i]) * stride[i];
        add(0, x, col, g.loc[((size_t)i * nl + dig[i]) * nl + y]);
        for (int t = 0; t < nterm; ++t)
          if (g.ctrl_node[t] == i) add(1 + g.term_ctrl[t], x, col, g.ctrl[((size_t)t * nl + dig[i]) * nl + y]);
      }
    for (const Pair &q : g.pairs) {
      const int xd = dig[q.dst], xs = dig[q.src];
      const bool rd = q.kind != 1, rs = q.kind == 2;        // raise the dst / src node?
      const cd vd = rd ? ra_val[xd] : lo_val[xd], vs = rs ? ra_val[xs] : lo_val[xs];
      if (vd == 0.0 || vs == 0.0 || q.dst == q.src) continue;
      const long long col = x + (long long)(rd ? ra_dl[xd] : lo_dl[xd]) * stride[q.dst] +
                            (long long)(rs ? ra_dl[xs] : lo_dl[xs]) * stride[q.src];
      add(0, x, col, q.coef * vd * vs);
    }
  }
  // Hermitian (h) and anti-Hermitian (a) parts, per row: |diagonal|-range and off-diagonal sums
  std::vector<double> hc(d, 0.0), hspread(d, 0.0), hrad(d, 0.0), arad(d, 0.0);
  for (int m = 0; m <= nc; ++m) {
    const double w = m == 0 ? 1.0 : E;
    std::unordered_map<long long, cd> herm, anti;
    for (const auto &kv : mats[m]) {
      const long long x = kv.first / d, y = kv.first % d;
      const cd v = kv.second;
      herm[x * d + y] += 0.5 * v;
      herm[y * d + x] += 0.5 * std::conj(v);
      anti[x * d + y] += v / cd(0.0, 2.0);
      anti[y * d + x] -= std::conj(v) / cd(0.0, 2.0);
    }
    for (const auto &kv : herm) {
      const long long x = kv.first / d, y = kv.first % d;
      if (x == y) {
        if (m == 0) hc[x] += kv.second.real();
        else hspread[x] += w * std::abs(kv.second.real());
      } else {
        hrad[x] += w * std::abs(kv.second);
      }
    }
    for (const auto &kv : anti) arad[kv.first / d] += w * std::abs(kv.second);   // diagonal counted too
  }
  Bounds b{1e300, -1e300, 0.0};
  for (int x = 0; x < d; ++x) {
    b.lo = std::min(b.lo, hc[x] - hspread[x] - hrad[x]);
    b.hi = std::max(b.hi, hc[x] + hspread[x] + hrad[x]);
    b.damp = std::max(b.damp, arad[x]);
  }
  return b;
}

}  // namespace

kt_status kt_fail(kt_status s, const char *msg) { return fail(s, "%s", msg); }

// ---------------------------------------------------------------------------- problem object
struct kt_problem {
  KtGeom g{};
  int fp64 = 1, ept = 4, cross = 0, density = 0;
  size_t esz = 16;
  // trajectory sharding: this problem holds trajectories [traj_offset, traj_offset + M) of M_total,
  // tiles [tile_off, tile_off + n_tiles) of n_tiles_total; the per-interval update sums the tile
  // partials of every shard, exchanged into gpart (all-gather over NCCL, or copies within a group)
  int sharded = 0, tile_off = 0, n_tiles_total = 0, M_total = 0;
  double *spart = nullptr;      // [n_tiles_total][n_ctrl]
  void *nccl_comm = nullptr;
  int nccl_rank = 0, nccl_world = 1;
  KtCplx *tau_all = nullptr;    // NCCL shards: tau of all M_total trajectories after a sweep
  bool in_group = false;
  int nt = 0, M = 0, n_passes = 0, n_passes_alloc = 0, ckpt = 0;
  int ckpt_dense = 0;           // ckpt > 0: co-states t_0 .. t_A all kept (A = ckpt_dense), then every ckpt-th
  bool ckpt_auto = false;       // storage chosen from free device memory (ckpt_interval = -1)
  double T = 0.0;
  size_t state_bytes = 0;       // one tile-layout array of all trajectories
  size_t bytes = 0;
  double e_min = 0, e_max = 0, damping = 0;
  std::vector<double> shape_h, lam_h;

  KtGenImage im_fwd{}, im_bwd{};
  KtOps ops{};
  std::vector<void *> allocs;

  double *eps_old = nullptr, *eps_new = nullptr, *deps = nullptr, *shape = nullptr, *U = nullptr;
  void *psi_init = nullptr, *psi[2] = {nullptr, nullptr};
  void *chi = nullptr;          // ckpt == 0: [nt+1] states, else the kept prefix and the checkpoints
  int n_chi_slots = 0;
  void *seg = nullptr;          // ckpt > 0: [ckpt + 1] states (segment / running buffers)
  double *rstate = nullptr;
  int *jcount[2] = {nullptr, nullptr}, *rec_step[2] = {nullptr, nullptr}, *rec_ch[2] = {nullptr, nullptr};
  double *rec_s[2] = {nullptr, nullptr}, *rec_c[2] = {nullptr, nullptr};
  int cur = 0;                  // record buffer written by a running forward sweep; 1-cur = last completed
  int *cursor = nullptr;
  double *partials = nullptr;
  unsigned *counter = nullptr;
  // whole-sweep launches (kt_config.per_interval_launches): sync = the grid barrier's two words
  int whole_sweep = 0;
  unsigned *sync = nullptr;
  KtCplx *tau = nullptr;
  double *norm2 = nullptr;
  int *status = nullptr;

  int *pass = nullptr;          // device [3]: next uniforms row, rows held, row of the running pass
  long long passes = 0;         // completed forward sweeps since the uniforms were uploaded
  long long sweeps = 0;         // completed forward sweeps since krotov_init (never reset)
  double *nu = nullptr;         // device [KT_MAX_CTRL]: pulse noise (krotov_pulse_noise)
  void *cwork = nullptr;        // cross-trajectory update: [x][k] states and control products
  double *cpart = nullptr;      // its per-tile partial sums
  double *cpair = nullptr;      // its per-slice pair sums
  unsigned *ccounter = nullptr;
  double *nu_ref = nullptr;     // device [n_ctrl][nt]: its reference pulse
  double *eps_base = nullptr;   // the pulse buffer eps_old pointed to at init (keys the graphs)
  bool have_fwd = false, have_bwd = false;
  int final_buf = 0;

  // gradient (krotov_gradient): forward states kept every Kg intervals, replayed per segment
  int Kg = 0, grad_ept = 4;
  KtGeom g1{};                  // the geometry re-cut to one trajectory per CTA
  void *psi_ck = nullptr;       // [nt/Kg + 1] states: psi(t_{s Kg}), s >= 1 (s = 0 is psi_init)
  void *psi_seg = nullptr;      // [Kg] replayed states of one segment
  void *chi_run[2] = {nullptr, nullptr};
  double *gpart = nullptr, *dgrad = nullptr;
  int *fcursor = nullptr;
  bool grad_ready = false;

  // optional per-launch timing of the interval kernels (krotov_set_profiling)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;            // pairs: [2i] before, [2i+1] after launch i
  std::vector<int> ev_family;                  // kernel family of pending pair i
  int ev_used = 0;
  double prof_ms[KT_PROF_FAMILIES] = {};
  long long prof_launches[KT_PROF_FAMILIES] = {};

  // Krotov iterations (backward sweep + updating forward sweep) captured as CUDA graphs, one per
  // buffer state: the record buffer being written (cur) and which pulse buffer holds the old pulse.
  // Both flip every iteration, so a run alternates between two of the four.
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t iter_graph[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t iter_exec[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

// In-place all-gather of equal slices over the shard communicator (a shard's own slice is already
// in place at its rank's offset).
kt_status nccl_allgather(kt_problem *p, const void *send, void *recv, size_t count, cudaStream_t st) {
  if (!p->nccl_comm) return fail(KT_ERR_STATE, "no NCCL communicator");
  const int r = g_nccl.all_gather(send, recv, count, kNcclDouble, p->nccl_comm, st);
  if (r != 0) return fail(KT_ERR_CUDA, "ncclAllGather failed: %s", g_nccl.error_string(r));
  return KT_OK;
}

// Event pair around one launch of the given family (only while profiling).
kt_status prof_begin(kt_problem *p, int family, cudaStream_t st) {
  if (!p->profiling) return KT_OK;
  const size_t need = 2 * (size_t)(p->ev_used + 1);
  while (p->ev_pool.size() < need) {
    cudaEvent_t e;
    KT_CUDA(cudaEventCreate(&e));
    p->ev_pool.push_back(e);
  }
  if (p->ev_family.size() < (size_t)p->ev_used + 1) p->ev_family.resize(p->ev_used + 1);
  p->ev_family[p->ev_used] = family;
  KT_CUDA(cudaEventRecord(p->ev_pool[2 * p->ev_used], st));
  return KT_OK;
}
kt_status prof_end(kt_problem *p, cudaStream_t st) {
  if (!p->profiling) return KT_OK;
  KT_CUDA(cudaEventRecord(p->ev_pool[2 * p->ev_used + 1], st));
  p->ev_used++;
  return KT_OK;
}
// After the stream has been synchronised: fold the pending pairs into the totals.
kt_status prof_collect(kt_problem *p) {
  for (int i = 0; i < p->ev_used; ++i) {
    float ms = 0.f;
    KT_CUDA(cudaEventElapsedTime(&ms, p->ev_pool[2 * i], p->ev_pool[2 * i + 1]));
    p->prof_ms[p->ev_family[i]] += ms;
    p->prof_launches[p->ev_family[i]] += 1;
  }
  p->ev_used = 0;
  return KT_OK;
}

kt_status dev_alloc(kt_problem *p, void **ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail(KT_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  p->bytes += bytes;
  return KT_OK;
}

template <typename T>
kt_status upload(kt_problem *p, T **dst, const T *src, size_t n, cudaStream_t st) {
  kt_status s = dev_alloc(p, (void **)dst, n * sizeof(T));
  if (s != KT_OK) return s;
  if (n) KT_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, st));
  return KT_OK;
}

void *state_slot(const kt_problem *p, void *base, long long slot) {
  return (char *)base + (size_t)slot * p->state_bytes;
}

// Co-state storage: ckpt == 0 keeps chi(t_j) for every j in slot j.  Otherwise slots 0..A hold
// chi(t_0)..chi(t_A) (A = ckpt_dense, possibly 0), then one slot per checkpoint t_{A + mK}
// (K = ckpt), and the last slot holds chi(t_nt); the co-states in between are recomputed segment
// by segment before the forward sweep needs them.
void *ckpt_slot(const kt_problem *p, int j) {
  if (p->ckpt == 0 || j <= p->ckpt_dense) return state_slot(p, p->chi, j);
  if (j == p->nt) return state_slot(p, p->chi, p->n_chi_slots - 1);
  return state_slot(p, p->chi, p->ckpt_dense + (j - p->ckpt_dense) / p->ckpt);
}
bool is_ckpt(const kt_problem *p, int j) {
  return p->ckpt == 0 || j <= p->ckpt_dense || j == p->nt || (j - p->ckpt_dense) % p->ckpt == 0;
}
int n_ckpt_slots(int nt, int A, int K) { return K == 0 ? nt + 1 : A + 1 + (nt - A + K - 1) / K; }
// End of the forward-sweep segment that starts at seg_a: the kept prefix is one segment (nothing to
// recompute), then checkpoint to checkpoint.
int seg_end(const kt_problem *p, int seg_a) {
  if (p->ckpt == 0) return p->nt;
  if (seg_a < p->ckpt_dense) return p->ckpt_dense;
  return std::min(seg_a + p->ckpt, p->nt);
}

kt_status read_status(kt_problem *p, cudaStream_t st) {
  int s = 0;
  KT_CUDA(cudaMemcpyAsync(&s, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  KT_CUDA(cudaStreamSynchronize(st));
  if (p->profiling) {
    kt_status ps = prof_collect(p);
    if (ps != KT_OK) return ps;
  }
  if (s == KT_DEV_OK) return KT_OK;
  KT_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), st));
  // a CTA that left early (a wait that ran out) took no last-CTA ticket: start the next sweep at zero
  KT_CUDA(cudaMemsetAsync(p->counter, 0, sizeof(unsigned), st));
  if (p->sync) KT_CUDA(cudaMemsetAsync(p->sync, 0, 2 * sizeof(unsigned), st));
  KT_CUDA(cudaStreamSynchronize(st));
  switch (s) {
    case KT_DEV_NONFINITE: return fail(KT_ERR_NONFINITE, "non-finite norm, overlap or pulse value on the device");
    case KT_DEV_RECORD_FULL: return fail(KT_ERR_RECORD_FULL, "a trajectory needed more jumps than draws_per_traj allows");
    case KT_DEV_RANGE: return fail(KT_ERR_RANGE, "a pulse value (updated, or set from device memory) left [-eps_bound, eps_bound]");
    case KT_DEV_ZERO_JUMP: return fail(KT_ERR_NONFINITE, "jump into a zero state (||L psi|| = 0 at a jump)");
    case KT_DEV_TIMEOUT: return fail(KT_ERR_TIMEOUT, "a bounded device-side wait for a bulk copy expired");
    default: return fail(KT_ERR_CUDA, "device status %d", s);
  }
}

FwdArgs fwd_args(kt_problem *p, int update) {
  FwdArgs a{};
  a.nt = p->nt;
  a.update = update;
  a.pass_row = p->pass + 2;
  a.overlap = update && !p->cross;
  a.eps_old = p->eps_old;
  a.eps_new = p->eps_new;
  a.deps = p->deps;
  a.shape = p->shape;
  a.U = p->U;
  a.rstate = p->rstate;
  a.jcount = p->jcount[p->cur];
  a.rec_step = p->rec_step[p->cur];
  a.rec_ch = p->rec_ch[p->cur];
  a.rec_s = p->rec_s[p->cur];
  a.rec_c = p->rec_c[p->cur];
  a.partials = p->sharded ? p->spart + (size_t)p->tile_off * p->g.n_ctrl : p->partials;
  a.finish = p->sharded ? 0 : 1;
  a.counter = p->counter;
  a.tau = p->tau;
  a.norm2 = p->norm2;
  a.status = p->status;
  return a;
}

BwdArgs bwd_args(kt_problem *p) {
  const int prev = 1 - p->cur;
  BwdArgs b{};
  b.nt = p->nt;
  b.eps = p->eps_old;
  b.cursor = p->cursor;
  b.advance_cursor = 1;
  b.forward_replay = 0;
  b.jcount = p->jcount[prev];
  b.rec_step = p->rec_step[prev];
  b.rec_ch = p->rec_ch[prev];
  b.rec_s = p->rec_s[prev];
  b.rec_c = p->rec_c[prev];
  b.status = p->status;
  return b;
}

kt_status launch_bwd_step(kt_problem *p, int j, const void *in, void *out, cudaStream_t st) {
  BwdArgs b = bwd_args(p);
  b.j = j;
  b.chi_in = in;
  b.chi_out = out;
  kt_status s = prof_begin(p, KT_PROF_BWD, st);
  if (s != KT_OK) return s;
  KT_CUDA(kt_launch_bwd(p->fp64, p->ept, p->g, p->im_bwd, p->ops, b, st));
  return prof_end(p, st);
}

// Recompute chi(t_{a+1}) .. chi(t_{b-1}) into seg[1 .. b-a-1] from the checkpoint at t_b.
kt_status recompute_segment(kt_problem *p, int a, int b, cudaStream_t st) {
  const int prev = 1 - p->cur;
  KT_CUDA(kt_launch_cursor_seek(p->g, p->rec_step[prev], p->jcount[prev], b, p->cursor, st));
  const void *in = ckpt_slot(p, b);
  for (int j = b; j >= a + 2; --j) {
    void *out = state_slot(p, p->seg, j - 1 - a);
    kt_status s = launch_bwd_step(p, j, in, out, st);
    if (s != KT_OK) return s;
    in = out;
  }
  return KT_OK;
}

const void *chi_at(const kt_problem *p, int j, int seg_a) {
  if (is_ckpt(p, j)) return ckpt_slot(p, j);
  return state_slot(p, p->seg, j - seg_a);
}

// Cross-trajectory update of interval j+1 from psi(t_j) and xi(t_j).
kt_status launch_cross(kt_problem *p, int j, const void *psi, const void *xi, cudaStream_t st) {
  const KtGeom &g = p->g;
  const size_t Mp = (size_t)(g.M + 31) / 32 * 32, n = (size_t)g.d * Mp;
  CrossArgs c{};
  c.j = j;
  c.nt = p->nt;
  c.psi = psi;
  c.xi = xi;
  c.X = p->cwork;
  c.P = (char *)p->cwork + n * p->esz;
  c.HP = (char *)p->cwork + 2 * n * p->esz;
  c.pairbuf = p->cpair;
  c.partials = p->cpart;
  c.counter = p->ccounter;
  c.eps_old = p->eps_old;
  c.eps_new = p->eps_new;
  c.deps = p->deps;
  c.shape = p->shape;
  c.status = p->status;
  kt_status s = prof_begin(p, KT_PROF_CROSS, st);
  if (s != KT_OK) return s;
  KT_CUDA(kt_launch_cross(p->fp64, g, p->ops, c, st));
  return prof_end(p, st);
}

// Start of the forward-sweep segment holding interval j (1-based): the kept prefix [0, A] is one
// segment, then checkpoint to checkpoint (see seg_end).
int seg_start(const kt_problem *p, int j) {
  if (p->ckpt == 0 || j <= p->ckpt_dense) return 0;
  return p->ckpt_dense + ((j - 1 - p->ckpt_dense) / p->ckpt) * p->ckpt;
}

// First launches of a forward sweep: the pass set-up and, for an updating sweep, the overlap at t_0
// (Delta eps of interval 1).
kt_status fwd_begin(kt_problem *p, int update, cudaStream_t st, FwdArgs &a) {
  KT_CUDA(kt_launch_init_pass(p->g, p->U, p->pass, p->rstate, p->jcount[p->cur], st));
  a = fwd_args(p, update);
  if (update && p->cross) {
    kt_status s = launch_cross(p, 0, p->psi_init, ckpt_slot(p, 0), st);
    if (s != KT_OK) return s;
  } else if (update) {
    a.j = 0;
    a.psi_in = p->psi_init;
    a.psi_out = nullptr;
    a.chi_t = ckpt_slot(p, 0);
    kt_status s = prof_begin(p, KT_PROF_FWD, st);
    if (s != KT_OK) return s;
    KT_CUDA(kt_launch_fwd(p->fp64, p->ept, p->g, p->im_fwd, p->ops, a, st));
    if ((s = prof_end(p, st)) != KT_OK) return s;
  }
  return KT_OK;
}

// Interval j of a forward sweep (with the co-state recompute of its segment first, if any).
kt_status fwd_step(kt_problem *p, int update, cudaStream_t st, bool save_psi, FwdArgs &a, int j) {
  const int seg_a = seg_start(p, j);
  kt_status s;
  if (update && p->ckpt > 0 && seg_a >= p->ckpt_dense && j == seg_a + 1 &&
      (s = recompute_segment(p, seg_a, seg_end(p, seg_a), st)) != KT_OK)
    return s;
  a.j = j;
  a.psi_in = (j == 1) ? p->psi_init : p->psi[(j - 1) & 1];
  a.psi_out = p->psi[j & 1];
  a.chi_t = (update && j < p->nt) ? chi_at(p, j, seg_a) : nullptr;
  if ((s = prof_begin(p, KT_PROF_FWD, st)) != KT_OK) return s;
  KT_CUDA(kt_launch_fwd(p->fp64, p->ept, p->g, p->im_fwd, p->ops, a, st));
  if ((s = prof_end(p, st)) != KT_OK) return s;
  if (update && p->cross && j < p->nt && (s = launch_cross(p, j, p->psi[j & 1], chi_at(p, j, seg_a), st)) != KT_OK)
    return s;
  if (save_psi && j < p->nt && j % p->Kg == 0)
    KT_CUDA(cudaMemcpyAsync(state_slot(p, p->psi_ck, j / p->Kg), p->psi[j & 1], p->state_bytes,
                            cudaMemcpyDeviceToDevice, st));
  return KT_OK;
}

// Sharded update of interval j+1 after the shards' overlaps at t_j are in spart: Delta eps from the
// partials of all tiles, in the single-GPU summation order.
kt_status shard_finish(kt_problem *p, int j, cudaStream_t st) {
  kt_status s = prof_begin(p, KT_PROF_FINISH, st);
  if (s != KT_OK) return s;
  KT_CUDA(kt_launch_finish_update(p->g, p->n_tiles_total, p->spart, j, p->nt, p->shape, p->eps_old, p->deps,
                                  p->eps_new, p->status, st));
  return prof_end(p, st);
}

// Launches of one forward sweep: no synchronisation and no change of host state, so that the
// sequence can be captured into a graph.  A shard driven by NCCL exchanges the tile partials of
// every interval (in-place all-gather) and, at the end, tau of all trajectories.
kt_status enqueue_forward(kt_problem *p, int update, cudaStream_t st, bool save_psi) {
  if (p->sharded && !p->nccl_comm)
    return fail(KT_ERR_STATE, "a trajectory shard runs through its group (krotov_group_update) or over NCCL "
                              "(krotov_shard_nccl)");
  if (p->whole_sweep && !save_psi) {
    // the whole sweep as one cooperative launch: interval 0 (the update overlap at t_0) when
    // updating, then 1 .. nt, psi(t_j) in psi[j & 1] as on the per-interval path
    KT_CUDA(kt_launch_init_pass(p->g, p->U, p->pass, p->rstate, p->jcount[p->cur], st));
    FwdArgs a = fwd_args(p, update);
    a.sweep = 1;
    a.j = (update && !p->cross) ? 0 : 1;
    a.psi_in = p->psi_init;
    a.psi_out = nullptr;
    a.psi_ring[0] = p->psi[0];
    a.psi_ring[1] = p->psi[1];
    a.chi_slots = p->chi;
    a.slot_bytes = p->state_bytes;
    a.sync = p->sync;
    KT_CUDA(cudaMemsetAsync(p->sync, 0, 2 * sizeof(unsigned), st));
    kt_status s = prof_begin(p, KT_PROF_FWD, st);
    if (s != KT_OK) return s;
    KT_CUDA(kt_launch_fwd(p->fp64, p->ept, p->g, p->im_fwd, p->ops, a, st));
    return prof_end(p, st);
  }
  FwdArgs a;
  kt_status s = fwd_begin(p, update, st, a);
  if (s != KT_OK) return s;
  const bool exchange = p->sharded && update && !p->cross;
  const size_t nloc = (size_t)p->g.n_tiles * p->g.n_ctrl;
  for (int j = 0; j <= p->nt; ++j) {
    if (j >= 1 && (s = fwd_step(p, update, st, save_psi, a, j)) != KT_OK) return s;
    if (exchange && j < p->nt) {
      if ((s = nccl_allgather(p, p->spart + (size_t)p->tile_off * p->g.n_ctrl, p->spart, nloc, st)) != KT_OK) return s;
      if ((s = shard_finish(p, j, st)) != KT_OK) return s;
    }
  }
  if (p->sharded && (s = nccl_allgather(p, p->tau, p->tau_all, (size_t)2 * p->M, st)) != KT_OK) return s;
  return KT_OK;
}

// Host bookkeeping of a completed forward sweep.
void commit_forward(kt_problem *p, int update, bool save_psi) {
  p->passes++;
  p->sweeps++;
  p->final_buf = p->nt & 1;
  if (update) std::swap(p->eps_old, p->eps_new);
  p->cur = 1 - p->cur;          // the records just written become the "last completed" ones
  p->have_fwd = true;
  p->have_bwd = false;
  p->grad_ready = save_psi;
}

kt_status forward_sweep(kt_problem *p, int update, cudaStream_t st, bool save_psi = false) {
  if (update && !p->have_bwd)
    return fail(KT_ERR_STATE, "an updating forward sweep needs a backward sweep since the last forward sweep");
  kt_status s = enqueue_forward(p, update, st, save_psi);
  if (s != KT_OK) return s;
  if ((s = read_status(p, st)) != KT_OK) return s;
  commit_forward(p, update, save_psi);
  return KT_OK;
}

// Buffers and geometry of the gradient sweep (first use only).
kt_status grad_setup(kt_problem *p, cudaStream_t st) {
  if (p->psi_ck) return KT_OK;
  if (p->density) return fail(KT_ERR_UNSUPPORTED, "the frozen-record gradient is defined for trajectory problems");
  KtGeom g1 = p->g;
  g1.T = 1;
  g1.n_tiles = p->M;
  g1.M_pad = p->M;
  g1.tile_elems = (g1.d + 3) / 4 * 4;
  g1.prefetch_chi = 0;
  // cavity structure with real / imaginary coupling classes, n_loc = 9, up to 96 fibers (the
  // compiled block size): one thread per last-node fiber; otherwise 4 items per thread up to 256
  // threads, else 8 up to 1024
  int ept;
  if ((p->ept == -309 || p->ept == -409) && g1.d / 9 <= 96) {
    ept = -409;
    g1.nthreads = std::max(32, (g1.d / 9 + 31) / 32 * 32);
  } else {
    ept = (g1.d + 3) / 4 <= 256 ? 4 : 8;
    if ((g1.d + ept - 1) / ept > 1024) return fail(KT_ERR_UNSUPPORTED, "dimension too large for the gradient kernel");
    g1.nthreads = std::max(32, ((g1.d + ept - 1) / ept + 31) / 32 * 32);
  }
  if (kt_grad_smem_bytes(g1, (int)p->esz) > 227 * 1024)
    return fail(KT_ERR_UNSUPPORTED, "the gradient needs four state buffers of d = %d in shared memory (%s)", g1.d,
                p->fp64 ? "use FP32-mixed" : "too large");
  p->g1 = g1;
  p->grad_ept = ept;
  // forward states kept every Kg intervals: the co-state spacing if one was given; with automatic
  // storage Kg ~ sqrt(nt), the fewest kept states (nt/Kg + Kg) for the same replay cost (about one
  // forward sweep whatever Kg > 1)
  if (p->ckpt_auto) p->Kg = std::max(1, (int)std::lround(std::sqrt((double)p->nt)));
  else p->Kg = p->ckpt > 0 ? p->ckpt : p->nt;
  kt_status s;
  if ((s = dev_alloc(p, &p->psi_ck, p->state_bytes * (p->nt / p->Kg + 1))) != KT_OK) return s;
  if ((s = dev_alloc(p, &p->psi_seg, p->state_bytes * p->Kg)) != KT_OK) return s;
  if ((s = dev_alloc(p, &p->chi_run[0], p->state_bytes)) != KT_OK) return s;
  if ((s = dev_alloc(p, &p->chi_run[1], p->state_bytes)) != KT_OK) return s;
  if ((s = dev_alloc(p, (void **)&p->gpart, (size_t)p->M * p->g.n_ctrl * sizeof(double))) != KT_OK) return s;
  if ((s = dev_alloc(p, (void **)&p->dgrad, (size_t)p->g.n_ctrl * p->nt * sizeof(double))) != KT_OK) return s;
  if ((s = dev_alloc(p, (void **)&p->fcursor, (size_t)p->g.M_pad * sizeof(int))) != KT_OK) return s;
  KT_CUDA(cudaMemsetAsync(p->dgrad, 0, (size_t)p->g.n_ctrl * p->nt * sizeof(double), st));
  return KT_OK;
}

// state psi(t_j) of the recorded forward pass inside segment [a, b): checkpoint or replayed
const void *psi_at(const kt_problem *p, int j, int seg_a) {
  if (j == seg_a) return seg_a == 0 ? p->psi_init : state_slot(p, p->psi_ck, seg_a / p->Kg);
  return state_slot(p, p->psi_seg, j - seg_a - 1);
}

// dJ_T/deps of the last (mode 2) forward sweep with its jump record frozen.
kt_status gradient_sweep(kt_problem *p, cudaStream_t st) {
  if (!p->grad_ready) return fail(KT_ERR_STATE, "krotov_gradient needs propagate_forward(p, 2, ...) first");
  const int prev = 1 - p->cur;
  KT_CUDA(kt_launch_chi_grad_boundary(p->fp64, p->g, p->ops, p->tau, p->norm2, p->psi[p->final_buf],
                                      p->chi_run[p->nt & 1], st));
  KT_CUDA(kt_launch_cursor_seek(p->g, p->rec_step[prev], p->jcount[prev], p->nt, p->cursor, st));
  GradArgs ga{};
  ga.nt = p->nt;
  ga.eps = p->eps_old;
  ga.cursor = p->cursor;
  ga.rec_step = p->rec_step[prev];
  ga.rec_ch = p->rec_ch[prev];
  ga.rec_s = p->rec_s[prev];
  ga.rec_c = p->rec_c[prev];
  ga.partials = p->gpart;
  ga.counter = p->counter;
  ga.grad = p->dgrad;
  ga.status = p->status;
  for (int seg_b = p->nt; seg_b > 0;) {
    const int seg_a = ((seg_b - 1) / p->Kg) * p->Kg;
    if (seg_b - 1 > seg_a) {
      KT_CUDA(kt_launch_cursor_seek_fwd(p->g, p->rec_step[prev], p->jcount[prev], seg_a + 1, p->fcursor, st));
      for (int j = seg_a + 1; j <= seg_b - 1; ++j) {
        BwdArgs b = bwd_args(p);
        b.j = j;
        b.chi_in = psi_at(p, j - 1, seg_a);
        b.chi_out = (void *)psi_at(p, j, seg_a);
        b.cursor = p->fcursor;
        b.forward_replay = 1;
        b.jcount = p->jcount[prev];
        kt_status s = prof_begin(p, KT_PROF_BWD, st);
        if (s != KT_OK) return s;
        KT_CUDA(kt_launch_bwd(p->fp64, p->ept, p->g, p->im_fwd, p->ops, b, st));
        if ((s = prof_end(p, st)) != KT_OK) return s;
      }
    }
    for (int j = seg_b; j >= seg_a + 1; --j) {
      ga.j = j;
      ga.psi_prev = psi_at(p, j - 1, seg_a);
      ga.chi_t = p->chi_run[j & 1];
      kt_status s = prof_begin(p, KT_PROF_GRAD, st);
      if (s != KT_OK) return s;
      KT_CUDA(kt_launch_grad(p->fp64, p->grad_ept, p->g1, p->g.T, p->g.tile_elems, p->im_fwd, p->im_bwd, p->ops, ga, st));
      if ((s = prof_end(p, st)) != KT_OK) return s;
      s = launch_bwd_step(p, j, p->chi_run[j & 1], p->chi_run[(j - 1) & 1], st);
      if (s != KT_OK) return s;
    }
    seg_b = seg_a;
  }
  return read_status(p, st);
}

// Launches of one backward sweep (capturable, like enqueue_forward).
kt_status enqueue_backward(kt_problem *p, cudaStream_t st) {
  const int prev = 1 - p->cur;
  void *chiT = ckpt_slot(p, p->nt);
  // chi_k(T) = tau_k |tgt>; the cross-trajectory xi_k(T) = |tgt>; a density matrix's P(T) = P_tgt
  KT_CUDA(kt_launch_chi_boundary(p->fp64, p->g, p->ops, (p->cross || p->density) ? nullptr : p->tau, chiT, st));
  KT_CUDA(kt_launch_cursor_seek(p->g, p->rec_step[prev], p->jcount[prev], p->nt, p->cursor, st));
  if (p->whole_sweep) {
    // the whole sweep as one launch: chi(t_{j-1}) of interval j into co-state slot j-1
    BwdArgs b = bwd_args(p);
    b.j = p->nt;
    b.sweep = 1;
    b.chi_in = chiT;
    b.chi_out = nullptr;
    b.chi_slots = p->chi;
    b.slot_bytes = p->state_bytes;
    kt_status s = prof_begin(p, KT_PROF_BWD, st);
    if (s != KT_OK) return s;
    KT_CUDA(kt_launch_bwd(p->fp64, p->ept, p->g, p->im_bwd, p->ops, b, st));
    return prof_end(p, st);
  }
  const void *in = chiT;
  for (int j = p->nt; j >= 1; --j) {
    void *out;
    if (is_ckpt(p, j - 1)) out = ckpt_slot(p, j - 1);
    else out = state_slot(p, p->seg, (j - 1) & 1);
    kt_status s = launch_bwd_step(p, j, in, out, st);
    if (s != KT_OK) return s;
    in = out;
  }
  return KT_OK;
}

kt_status backward_sweep(kt_problem *p, cudaStream_t st) {
  if (!p->have_fwd) return fail(KT_ERR_STATE, "propagate_backward needs a forward sweep first");
  kt_status s = enqueue_backward(p, st);
  if (s != KT_OK) return s;
  if ((s = read_status(p, st)) != KT_OK) return s;
  p->have_bwd = true;
  return KT_OK;
}

int iter_key(const kt_problem *p) { return p->cur | (p->eps_old == p->eps_base ? 2 : 0); }

// Capture one Krotov iteration (backward sweep with the last records and the old pulse, then the
// updating forward sweep) for the current buffer state.  Capture runs on the problem's own
// stream, because the legacy default stream cannot be captured.
kt_status capture_iteration(kt_problem *p, cudaGraph_t *out) {
  const int key = iter_key(p);
  if (p->iter_graph[key]) {
    *out = p->iter_graph[key];
    return KT_OK;
  }
  if (!p->cap_stream) KT_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
  KT_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
  kt_status s = enqueue_backward(p, p->cap_stream);
  if (s == KT_OK) s = enqueue_forward(p, 1, p->cap_stream, false);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
  if (s != KT_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return s != KT_OK ? s : fail(KT_ERR_CUDA, "graph capture of a Krotov iteration failed: %s", cudaGetErrorString(e));
  }
  p->iter_graph[key] = graph;
  *out = graph;
  return KT_OK;
}

// Host bookkeeping of a completed graph iteration.
void commit_iteration(kt_problem *p) {
  p->have_bwd = true;
  commit_forward(p, 1, false);
}

// One Krotov iteration as a single graph launch on st.
kt_status graph_iteration(kt_problem *p, cudaStream_t st) {
  const int key = iter_key(p);
  if (!p->iter_exec[key]) {
    cudaGraph_t graph;
    kt_status s = capture_iteration(p, &graph);
    if (s != KT_OK) return s;
    KT_CUDA(cudaGraphInstantiate(&p->iter_exec[key], graph, 0));
  }
  KT_CUDA(cudaGraphLaunch(p->iter_exec[key], st));
  kt_status s = read_status(p, st);
  if (s != KT_OK) {
    p->have_fwd = p->have_bwd = false;    // the iteration's sweeps are incomplete: restart from a forward sweep
    return s;
  }
  commit_iteration(p);
  return KT_OK;
}

// F of the last forward sweep (a shard over NCCL: of all M_total trajectories, from the gathered tau,
// summed in trajectory order like the single-GPU problem); tau_out gets this problem's M values.
kt_status host_fidelity(kt_problem *p, double *F, double *tau_out, cudaStream_t st) {
  const bool all = p->sharded && p->nccl_comm;
  const int n = all ? p->M_total : p->M;
  std::vector<KtCplx> tau(n);
  KT_CUDA(cudaMemcpyAsync(tau.data(), all ? p->tau_all : p->tau, sizeof(KtCplx) * n, cudaMemcpyDeviceToHost, st));
  KT_CUDA(cudaStreamSynchronize(st));
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += tau[k].re * tau[k].re + tau[k].im * tau[k].im;
  if (F) *F = s / n;
  if (all && tau_out) {
    for (int k = 0; k < p->M; ++k) {
      tau_out[2 * k] = tau[p->tile_off * p->g.T + k].re;
      tau_out[2 * k + 1] = tau[p->tile_off * p->g.T + k].im;
    }
    return KT_OK;
  }
  if (F && p->density) *F = tau[0].re;        // <<P_tgt|rho(T)>> = <tgt|rho(T)|tgt>
  if (tau_out)
    for (int k = 0; k < p->M; ++k) {
      tau_out[2 * k] = tau[k].re;
      tau_out[2 * k + 1] = tau[k].im;
    }
  return KT_OK;
}

// Tile layout: trajectory k = tile*T + t, element x at tile*tile_elems + x*T + t.
template <typename R>
void to_tiles(const kt_problem *p, const double *src /*[M][d][2] or [d][2]*/, bool batch, std::vector<R> &out) {
  const KtGeom &g = p->g;
  out.assign((size_t)g.n_tiles * g.tile_elems * 2, (R)0);
  for (int k = 0; k < g.M; ++k) {
    const double *v = batch ? src + (size_t)k * g.d * 2 : src;
    const int tile = k / g.T, t = k % g.T;
    for (int x = 0; x < g.d; ++x) {
      const size_t e = (size_t)tile * g.tile_elems + (size_t)x * g.T + t;
      out[2 * e] = (R)v[2 * x];
      out[2 * e + 1] = (R)v[2 * x + 1];
    }
  }
}

kt_status download_state(kt_problem *p, const void *dev, double *out, cudaStream_t st) {
  const KtGeom &g = p->g;
  std::vector<char> buf(p->state_bytes);
  KT_CUDA(cudaMemcpyAsync(buf.data(), dev, p->state_bytes, cudaMemcpyDeviceToHost, st));
  KT_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < g.M; ++k) {
    const int tile = k / g.T, t = k % g.T;
    for (int x = 0; x < g.d; ++x) {
      const size_t e = (size_t)tile * g.tile_elems + (size_t)x * g.T + t;
      double re, im;
      if (p->fp64) {
        re = ((const double *)buf.data())[2 * e];
        im = ((const double *)buf.data())[2 * e + 1];
      } else {
        re = ((const float *)buf.data())[2 * e];
        im = ((const float *)buf.data())[2 * e + 1];
      }
      out[((size_t)k * g.d + x) * 2] = re;
      out[((size_t)k * g.d + x) * 2 + 1] = im;
    }
  }
  return KT_OK;
}

int ipow(int b, int e) {
  long long r = 1;
  for (int i = 0; i < e; ++i) {
    r *= b;
    if (r > (1 << 30)) return -1;
  }
  return (int)r;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

KT_API const char *krotov_last_error(void) { return g_err.c_str(); }

KT_API kt_status kt_bessel_j(double alpha, int n, double *out) {
  if (!out) return fail(KT_ERR_ARG, "out is NULL");
  if (kt_bessel_miller(alpha, n, out) != 0) return fail(KT_ERR_ARG, "alpha must be >= 0 and n in [1, 256]");
  return KT_OK;
}

KT_API void krotov_free(kt_problem *p) {
  if (!p) return;
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (int k = 0; k < 4; ++k) {
    if (p->iter_exec[k]) cudaGraphExecDestroy(p->iter_exec[k]);
    if (p->iter_graph[k]) cudaGraphDestroy(p->iter_graph[k]);
  }
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->nccl_comm && g_nccl.comm_destroy) g_nccl.comm_destroy(p->nccl_comm);
  for (void *a : p->allocs) cudaFree(a);
  delete p;
}

}  // extern "C"

namespace {

// Everything krotov_init computes on the host, before any device call.
struct HostImage {
  std::vector<int> dl, poff;
  std::vector<KtCplx> base, cslot, dg, cdg, pval, cf, pc;
  int pdst[KT_MAX_PAIRS], psrc[KT_MAX_PAIRS];
  double kd[2 * KT_MAX_NL] = {}, kc[4] = {}, kp[KT_MAX_PAIRS] = {};   // constants of the real / imaginary kernels
};

struct HostPlan {
  KtGeom g{};
  int fp64 = 1, ept = 4, ckpt = 0, ckpt_dense = 0, cross = 0, density = 0;
  int sharded = 0, tile_off = 0, n_tiles_total = 0, M_total = 0;
  std::vector<double> psi0;    // density: vec(rho_0) [d][2]; empty otherwise (the model's psi0 is used)
  double e_min = 0, e_max = 0, damping = 0;
  HostImage fwd, bwd;
  std::vector<int> lo_dl, ra_dl, hc_dl;
  std::vector<KtCplx> lo_val, ra_val, lind, hc_val, tgt;
  std::vector<uint32_t> digits;
};

// True when the model has the node structure of the cascaded atom-cavity network (Sec. 3.1):
// local index atom * (nc+1) + n with atom in {g, e, r}, the ladder factor the cavity
// annihilation operator, and the last node's factor (both directions, drift and controls)
// coupling only (r, n-1) <-> (g, n) and (r, n) <-> (e, n) off the diagonal.  The kernels then
// take the cavity-structure fast path.
bool cavity_structure(const Gen &gf, const Gen &gb, const std::vector<int> &lo_dl, const std::vector<cd> &lo_val,
                      const std::vector<int> &ra_dl, const std::vector<cd> &ra_val) {
  const int nl = gf.nl;
  if (nl != 6 && nl != 9) return false;
  for (const Pair &q : gf.pairs)
    if (q.kind != 0) return false;           // the fast path's pair hops raise one node and lower the other
  const int NP = nl / 3, NC = NP - 1;
  for (int x = 0; x < nl; ++x) {
    const int n = x % NP;
    if ((lo_val[x] != 0.0) != (n < NC) || (n < NC && lo_dl[x] != 1)) return false;
    if ((ra_val[x] != 0.0) != (n >= 1) || (n >= 1 && ra_dl[x] != -1)) return false;
  }
  auto allowed = [&](int x, int y) {
    const int ax = x / NP, nx = x % NP, ay = y / NP, ny = y % NP;
    if (((ax == 1 && ay == 2) || (ax == 2 && ay == 1)) && nx == ny) return true;   // drive e <-> r
    if (ax == 2 && ay == 0 && ny == nx + 1) return true;                           // cavity (r,n-1) <- (g,n)
    if (ax == 0 && ay == 2 && nx == ny + 1) return true;                           // cavity (g,n) <- (r,n-1)
    return false;
  };
  const int last = gf.N - 1;
  auto check = [&](const std::vector<cd> &m, size_t base) {
    for (int x = 0; x < nl; ++x)
      for (int y = 0; y < nl; ++y)
        if (x != y && m[base + x * nl + y] != 0.0 && !allowed(x, y)) return false;
    return true;
  };
  if (!check(gf.loc, (size_t)last * nl * nl) || !check(gb.loc, (size_t)last * nl * nl)) return false;
  for (size_t c = 0; c < gf.ctrl_node.size(); ++c)
    if (gf.ctrl_node[c] == last && (!check(gf.ctrl, c * nl * nl) || !check(gb.ctrl, c * nl * nl))) return false;
  return true;
}

// The real / imaginary cavity-structure kernels take as constants the last node's diagonal and
// cavity couplings, the pair coefficients and the ladder values sqrt(n): true when no control term
// on the last node touches its diagonal or cavity couplings (those entries are then the same in every
// interval) and the ladder factor is the cavity annihilation operator, <n-1|a|n> = sqrt(n) exactly.
bool acs_constants_ok(const Gen &gf, const Gen &gb, const std::vector<cd> &lo_val, const std::vector<cd> &ra_val) {
  const int nl = gf.nl, NP = nl / 3, NC = NP - 1, last = gf.N - 1;
  for (int x = 0; x < nl; ++x) {
    const int n = x % NP;
    if (n < NC && lo_val[x] != cd(std::sqrt((double)(n + 1)), 0.0)) return false;
    if (n >= 1 && ra_val[x] != cd(std::sqrt((double)n), 0.0)) return false;
  }
  for (const Gen *gen : {&gf, &gb})
    for (size_t t = 0; t < gen->ctrl_node.size(); ++t) {
      if (gen->ctrl_node[t] != last) continue;
      for (int x = 0; x < nl; ++x)
        if (at(gen->ctrl, (int)t * nl * nl, nl, x, x) != 0.0) return false;
      for (int n = 1; n <= NC; ++n) {
        const int qr = 2 * NP + n - 1, qg = n;
        if (at(gen->ctrl, (int)t * nl * nl, nl, qr, qg) != 0.0 || at(gen->ctrl, (int)t * nl * nl, nl, qg, qr) != 0.0)
          return false;
      }
    }
  return true;
}

// Real / imaginary coupling classes, checked on top of the cavity structure: every off-diagonal
// entry of every node factor (drift and controls, both directions) is purely real or purely
// imaginary, a row has at most one entry of each class, the last node's cavity couplings are real
// and its drive couplings imaginary, every pair coefficient is imaginary and the ladder factor is
// real (true of the node of Sec. 3.1: g real, drive (i/2)(sigma_re - sigma_er), cascade -2i kappa).
// Then each row's slots are re-ordered [real entry, imaginary entry] (x itself marks an empty
// slot), and the kernels apply each coupling with two real FMAs instead of a complex one; the
// result is bit-identical, the products with the zero part being exact zeros.
bool ri_classes(const Gen &gf, const Gen &gb, const std::vector<cd> &lo_val, const std::vector<cd> &ra_val,
                std::vector<std::vector<int>> &cols) {
  const int N = gf.N, nl = gf.nl, NP = nl / 3;
  for (int x = 0; x < nl; ++x)
    if (lo_val[x].imag() != 0.0 || ra_val[x].imag() != 0.0) return false;
  for (const Gen *gen : {&gf, &gb})
    for (const Pair &q : gen->pairs)
      if (q.coef.real() != 0.0) return false;
  // 0: zero, 1: real, 2: imaginary, 3: neither
  auto cls = [&](int i, int x, int y) {
    bool re = false, im = false;
    auto take = [&](cd v) {
      if (v.real() != 0.0) re = true;
      if (v.imag() != 0.0) im = true;
    };
    take(at(gf.loc, i * nl * nl, nl, x, y));
    take(at(gb.loc, i * nl * nl, nl, x, y));
    for (size_t c = 0; c < gf.ctrl_node.size(); ++c)
      if (gf.ctrl_node[c] == i) {
        take(at(gf.ctrl, (int)c * nl * nl, nl, x, y));
        take(at(gb.ctrl, (int)c * nl * nl, nl, x, y));
      }
    return re && im ? 3 : re ? 1 : im ? 2 : 0;
  };
  std::vector<std::vector<int>> out(cols.size());
  for (int i = 0; i < N; ++i)
    for (int x = 0; x < nl; ++x) {
      int yr = x, yi = x;
      for (int y : cols[(size_t)i * nl + x]) {
        const int k = cls(i, x, y);
        if (k == 3) return false;
        if (k == 1) {
          if (yr != x) return false;
          yr = y;
        } else if (k == 2) {
          if (yi != x) return false;
          yi = y;
        }
      }
      if (i == N - 1 && yr != x && (x / NP) * (yr / NP) != 0) return false;   // cavity: g <-> r only
      if (i == N - 1 && yi != x && (x / NP) * (yi / NP) != 2) return false;   // drive: e <-> r only
      out[(size_t)i * nl + x] = {yr, yi};
    }
  cols.swap(out);
  return true;
}

// Validation, a1 (structured H_eff = H - (i/2) sum_l L_l^dag L_l), a2 (spectral interval and
// Chebyshev length), tile geometry and the scaled generator tables of both directions.
kt_status plan(const kt_model_desc *md, const kt_config *cfg, HostPlan &P, bool density = false) {
  if (!md || !cfg) return fail(KT_ERR_ARG, "NULL descriptor");
  int N = md->n_nodes;
  const int nl = md->n_loc;
  if (N < 1 || N > KT_MAX_NODES) return fail(KT_ERR_UNSUPPORTED, "n_nodes must be in [1, %d]", KT_MAX_NODES);
  if (nl < 2 || nl > 16) return fail(KT_ERR_UNSUPPORTED, "n_loc must be in [2, 16]");
  int d = ipow(nl, N);
  if (d < 0) return fail(KT_ERR_UNSUPPORTED, "dimension n_loc^n_nodes too large");
  if (md->n_ctrl < 1 || md->n_ctrl > KT_MAX_CTRL) return fail(KT_ERR_ARG, "n_ctrl must be in [1, %d]", KT_MAX_CTRL);
  if (md->n_lind < 0 || md->n_lind > KT_MAX_LIND) return fail(KT_ERR_ARG, "n_lind must be in [0, %d]", KT_MAX_LIND);
  if (md->n_pairs < 0) return fail(KT_ERR_ARG, "n_pairs < 0");
  if (!md->h0_local || !md->hc_local || !md->ctrl_node || !md->psi_tgt || (!md->psi0 && !md->psi0_batch))
    return fail(KT_ERR_ARG, "missing model arrays");
  if ((md->n_pairs > 0 || md->n_lind > 0) && !md->a_local) return fail(KT_ERR_ARG, "a_local required for pairs / Lindblad operators");
  if (md->n_pairs > 0 && (!md->pair_dst || !md->pair_src || !md->pair_coef)) return fail(KT_ERR_ARG, "missing pair arrays");
  if (md->n_lind > 0 && !md->lind_coef) return fail(KT_ERR_ARG, "missing lind_coef");
  if (cfg->nt < 1 || cfg->M < 1 || !(cfg->T > 0.0)) return fail(KT_ERR_ARG, "need nt >= 1, M >= 1, T > 0");
  if (!cfg->eps_guess || !cfg->shape || !cfg->lambda_a || !cfg->uniforms) return fail(KT_ERR_ARG, "missing config arrays");
  if (cfg->n_passes < 1 || cfg->draws_per_traj < 1 || cfg->draws_per_traj % 2 == 0)
    return fail(KT_ERR_ARG, "need n_passes >= 1 and odd draws_per_traj >= 1");
  if (cfg->prec != KT_FP64 && cfg->prec != KT_FP32_MIXED) return fail(KT_ERR_ARG, "unknown precision");
  if (cfg->ckpt_interval < -1) return fail(KT_ERR_ARG, "ckpt_interval must be -1 (automatic), 0 or > 0");
  if (cfg->tile_traj < -1) return fail(KT_ERR_ARG, "tile_traj must be -1 (autotuned), 0 (automatic) or a power of two <= 32");
  if (cfg->update_rule != 0 && cfg->update_rule != 1) return fail(KT_ERR_ARG, "update_rule must be 0 or 1");
  const bool sharded = cfg->M_total > 0;
  if (sharded) {
    if (cfg->traj_offset < 0 || cfg->traj_offset + cfg->M > cfg->M_total)
      return fail(KT_ERR_ARG, "a shard needs 0 <= traj_offset and traj_offset + M <= M_total");
    if (cfg->update_rule != 0 || density)
      return fail(KT_ERR_ARG, "sharding covers the independent-trajectory update (the cross-trajectory sum "
                              "needs every pair of trajectories)");
    if (cfg->tile_traj == -1) return fail(KT_ERR_ARG, "the shards of one problem need one tile width: no autotuning");
  } else if (cfg->traj_offset != 0) {
    return fail(KT_ERR_ARG, "traj_offset without M_total");
  }
  if (density && (cfg->update_rule != 0 || cfg->M != 1))
    return fail(KT_ERR_ARG, "a density-matrix problem has one Liouville-space state and the update of Eq. krotovupdate");
  if (cfg->jump_scheme != 0 && cfg->jump_scheme != 1) return fail(KT_ERR_ARG, "jump_scheme must be 0 or 1");
  for (int c = 0; c < md->n_ctrl; ++c) {
    if (md->ctrl_node[c] < 0 || md->ctrl_node[c] >= N) return fail(KT_ERR_ARG, "ctrl_node[%d] out of range", c);
    if (!(cfg->lambda_a[c] > 0.0)) return fail(KT_ERR_ARG, "lambda[%d] must be > 0", c);
  }
  const int nt = cfg->nt, M = cfg->M, nc = md->n_ctrl;
  for (long i = 0; i < (long)nc * nt; ++i)
    if (!std::isfinite(cfg->eps_guess[i]) || !std::isfinite(cfg->shape[i]))
      return fail(KT_ERR_NONFINITE, "non-finite guess pulse or shape value");

  // ---- a1
  Gen gf;
  gf.N = N;
  gf.nl = nl;
  gf.loc.assign((size_t)N * nl * nl, 0.0);
  for (size_t e = 0; e < gf.loc.size(); ++e) gf.loc[e] = cd(md->h0_local[2 * e], md->h0_local[2 * e + 1]);
  gf.ctrl.assign((size_t)nc * nl * nl, 0.0);
  for (size_t e = 0; e < gf.ctrl.size(); ++e) gf.ctrl[e] = cd(md->hc_local[2 * e], md->hc_local[2 * e + 1]);
  gf.ctrl_node.assign(md->ctrl_node, md->ctrl_node + nc);
  gf.n_ctrl = nc;
  for (int c = 0; c < nc; ++c) gf.term_ctrl.push_back(c);
  std::vector<cd> a(nl * nl, 0.0);
  if (md->a_local)
    for (int e = 0; e < nl * nl; ++e) a[e] = cd(md->a_local[2 * e], md->a_local[2 * e + 1]);
  double amax = 0.0;
  std::vector<int> lo_dl(nl, 0), ra_dl(nl, 0);
  std::vector<cd> lo_val(nl, 0.0), ra_val(nl, 0.0);
  for (int x = 0; x < nl; ++x) {
    int nr = 0, ncol = 0;
    for (int y = 0; y < nl; ++y) {
      if (a[x * nl + y] != 0.0) { ++nr; lo_dl[x] = y - x; lo_val[x] = a[x * nl + y]; }
      if (a[y * nl + x] != 0.0) { ++ncol; ra_dl[x] = y - x; ra_val[x] = std::conj(a[y * nl + x]); }
      amax = std::max(amax, std::abs(a[x * nl + y]));
    }
    if (nr > 1 || ncol > 1) return fail(KT_ERR_ARG, "a_local must have at most one nonzero per row and per column");
    if (a[x * nl + x] != 0.0 && (md->n_pairs > 0 || md->n_lind > 0))
      return fail(KT_ERR_ARG, "a_local must have no diagonal entry (a ladder factor moves the local state)");
  }
  std::vector<Pair> raw;
  for (int q = 0; q < md->n_pairs; ++q) {
    const int ds = md->pair_dst[q], sr = md->pair_src[q];
    if (ds < 0 || ds >= N || sr < 0 || sr >= N || ds == sr) return fail(KT_ERR_ARG, "bad pair %d", q);
    raw.push_back(Pair{ds, sr, cd(md->pair_coef[2 * q], md->pair_coef[2 * q + 1])});
  }
  const std::vector<cd> ada = adag_a(a, nl);
  for (int l = 0; l < md->n_lind; ++l)
    for (int i = 0; i < N; ++i)
      for (int jn = 0; jn < N; ++jn) {
        const cd ci = cd(md->lind_coef[2 * (l * N + i)], md->lind_coef[2 * (l * N + i) + 1]);
        const cd cj = cd(md->lind_coef[2 * (l * N + jn)], md->lind_coef[2 * (l * N + jn) + 1]);
        const cd w = cd(0.0, -0.5) * std::conj(ci) * cj;     // -(i/2) conj(c_i) c_j a_i^dag a_j
        if (w == 0.0) continue;
        if (i == jn) {
          for (int e = 0; e < nl * nl; ++e) gf.loc[(size_t)i * nl * nl + e] += w * ada[e];
        } else {
          raw.push_back(Pair{i, jn, w});
        }
      }
  double pmax = 1.0;
  for (const Pair &q : raw) pmax = std::max(pmax, std::abs(q.coef));
  for (const Pair &q : raw) {
    bool merged = false;
    for (Pair &o : gf.pairs)
      if (o.dst == q.dst && o.src == q.src) { o.coef += q.coef; merged = true; }
    if (!merged) gf.pairs.push_back(q);
  }
  // terms cancelled to rounding level (e.g. the upstream cascade hop) are dropped
  gf.pairs.erase(std::remove_if(gf.pairs.begin(), gf.pairs.end(),
                                [&](const Pair &q) { return std::abs(q.coef) <= 1e-13 * pmax; }),
                 gf.pairs.end());
  std::vector<cd> psi_t(d), psi_0;                        // target (and density: initial) state vectors
  for (int x = 0; x < d; ++x) psi_t[x] = cd(md->psi_tgt[2 * x], md->psi_tgt[2 * x + 1]);
  int n_lind = md->n_lind;
  if (density) {
    // Liouville space (Sec. 2.2, Eq. lindblad): rho_{xy} -> vec(rho)[x d + y] evolves as
    // d vec(rho)/dt = -i G vec(rho), G = H_eff (x) 1 - 1 (x) H_eff^* + i sum_l L_l (x) L_l^*, a network of
    // 2N nodes (ket nodes 0..N-1, bra nodes N..2N-1, same local dimension): the ket nodes carry
    // H_eff's factors and hops, the bra nodes minus their complex conjugates (the ladder factor is
    // real, so conj(a) = a), and every pair (ket i, bra j) the hop i c_li conj(c_lj) a_i a_j (kind 1).
    // A control eps_c acts through H_c (x) 1 - 1 (x) H_c^*: one term on its ket and one on its bra node.
    for (int e = 0; e < nl * nl; ++e)
      if (a[e].imag() != 0.0) return fail(KT_ERR_UNSUPPORTED, "density-matrix problems need a real ladder factor");
    if (2 * N > KT_MAX_NODES) return fail(KT_ERR_UNSUPPORTED, "density-matrix problems need n_nodes <= %d", KT_MAX_NODES / 2);
    Gen lg;
    lg.N = 2 * N;
    lg.nl = nl;
    lg.n_ctrl = nc;
    lg.loc.assign((size_t)2 * N * nl * nl, 0.0);
    for (int i = 0; i < N; ++i)
      for (int e = 0; e < nl * nl; ++e) {
        lg.loc[(size_t)i * nl * nl + e] = gf.loc[(size_t)i * nl * nl + e];
        lg.loc[(size_t)(N + i) * nl * nl + e] = -std::conj(gf.loc[(size_t)i * nl * nl + e]);
      }
    for (int c = 0; c < nc; ++c)
      for (int side = 0; side < 2; ++side) {
        for (int e = 0; e < nl * nl; ++e) {
          const cd v = gf.ctrl[(size_t)c * nl * nl + e];
          lg.ctrl.push_back(side == 0 ? v : -std::conj(v));
        }
        lg.ctrl_node.push_back(gf.ctrl_node[c] + side * N);
        lg.term_ctrl.push_back(c);
      }
    for (const Pair &q : gf.pairs) {
      lg.pairs.push_back(Pair{q.dst, q.src, q.coef, 0});
      lg.pairs.push_back(Pair{N + q.dst, N + q.src, -std::conj(q.coef), 0});
    }
    for (int i = 0; i < N; ++i)
      for (int jn = 0; jn < N; ++jn) {
        cd w = 0.0;
        for (int l = 0; l < md->n_lind; ++l) {
          const cd ci = cd(md->lind_coef[2 * (l * N + i)], md->lind_coef[2 * (l * N + i) + 1]);
          const cd cj = cd(md->lind_coef[2 * (l * N + jn)], md->lind_coef[2 * (l * N + jn) + 1]);
          w += cd(0.0, 1.0) * ci * std::conj(cj);
        }
        if (w != 0.0) lg.pairs.push_back(Pair{i, N + jn, w, 1});
      }
    const long long dd = (long long)d * d;
    if (dd > (1 << 24)) return fail(KT_ERR_UNSUPPORTED, "density-matrix problems need d^2 <= 2^24");
    std::vector<cd> psi0v(d);
    for (int x = 0; x < d; ++x) {
      if (!md->psi0) return fail(KT_ERR_ARG, "density-matrix problems start from the pure state psi0");
      psi0v[x] = cd(md->psi0[2 * x], md->psi0[2 * x + 1]);
    }
    psi_0.assign((size_t)dd, 0.0);
    std::vector<cd> vt((size_t)dd);
    for (int x = 0; x < d; ++x)
      for (int y = 0; y < d; ++y) {
        psi_0[(size_t)x * d + y] = psi0v[x] * std::conj(psi0v[y]);     // rho_0 = |psi0><psi0|
        vt[(size_t)x * d + y] = psi_t[x] * std::conj(psi_t[y]);         // P(T) = |tgt><tgt|
      }
    psi_t.swap(vt);
    gf = lg;
    N = 2 * N;
    d = (int)dd;
    n_lind = 0;                            // no jumps: the density matrix evolves deterministically
  }
  if ((int)gf.pairs.size() > KT_MAX_PAIRS) return fail(KT_ERR_UNSUPPORTED, "more than %d pair terms", KT_MAX_PAIRS);
  if ((int)gf.ctrl_node.size() > KT_MAX_CTERMS) return fail(KT_ERR_UNSUPPORTED, "more than %d control terms", KT_MAX_CTERMS);
  const Gen gb = minus_adjoint(gf);
  const int nterm = (int)gf.ctrl_node.size();

  // ---- a2
  double E = cfg->eps_bound;
  if (!(E > 0.0)) {
    double m = 0.0;
    for (long i = 0; i < (long)nc * nt; ++i) m = std::max(m, std::fabs(cfg->eps_guess[i]));
    E = 2.0 * m + 1.0;
  }
  for (long i = 0; i < (long)nc * nt; ++i)
    if (std::fabs(cfg->eps_guess[i]) > E) return fail(KT_ERR_RANGE, "guess pulse exceeds eps_bound");
  // spectral interval: the tighter of the per-node bounds and whole-row Gershgorin discs (rows
  // enumerated on the host, at most d = 2^22 of them)
  Bounds bf = gen_bounds(gf, amax, E), bb = gen_bounds(gb, amax, E);
  if (d <= (1 << 22)) {
    int strd[KT_MAX_NODES];
    for (int i = 0; i < N; ++i) strd[i] = ipow(nl, N - 1 - i);
    const Bounds rf = row_bounds(gf, lo_dl, lo_val, ra_dl, ra_val, d, strd, E);
    const Bounds rb{-rf.hi, -rf.lo, rf.damp};        // -G^dag: Hermitian part negated, same anti part
    if (rf.hi - rf.lo < bf.hi - bf.lo) { bf.lo = rf.lo; bf.hi = rf.hi; }
    if (rb.hi - rb.lo < bb.hi - bb.lo) { bb.lo = rb.lo; bb.hi = rb.hi; }
    bf.damp = std::min(bf.damp, rf.damp);
    bb.damp = std::min(bb.damp, rf.damp);
  }
  const double r = 0.5 * std::max(bf.hi - bf.lo, bb.hi - bb.lo) * 1.0001 + 1e-12;
  const double c_fwd = 0.5 * (bf.lo + bf.hi), c_bwd = 0.5 * (bb.lo + bb.hi);
  const double damp = std::max(bf.damp, bb.damp);
  const double dt = cfg->T / nt;
  const cd z(1.0, damp / r);
  const double rho = std::max(1.0, std::abs(z + std::sqrt(z - 1.0) * std::sqrt(z + 1.0)));
  // default truncation: 1e-16 in FP64 (the row bound is sharp, so the criterion's margin is the
  // tolerance itself), the FP32 unit roundoff 2^-24 in FP32-mixed (the truncation error then stays
  // an order of magnitude below the rounding the FP32 recurrence accumulates anyway)
  const double tol = cfg->cheb_tol > 0 ? cfg->cheb_tol : (cfg->prec == KT_FP64 ? 1e-16 : 0x1p-24);
  std::vector<double> J(256);
  kt_bessel_miller(r * dt, 256, J.data());
  int K = -1;
  for (int k = 1; k < 250; ++k) {
    bool small = true;
    for (int q = k; q < k + 6; ++q)
      if (std::fabs(J[q]) * std::pow(rho, q) >= tol) small = false;
    if (small && k > r * dt) { K = k; break; }
  }
  if (K < 1 || K > KT_MAX_K) return fail(KT_ERR_UNSUPPORTED, "Chebyshev series needs %d > %d terms (reduce dt)", K, KT_MAX_K);

  P.fp64 = cfg->prec == KT_FP64;
  P.cross = cfg->update_rule;
  P.ckpt = (cfg->ckpt_interval > 0 && cfg->ckpt_interval < nt) ? cfg->ckpt_interval : 0;
  if (cfg->ckpt_prefix < 0) return fail(KT_ERR_ARG, "ckpt_prefix < 0");
  P.ckpt_dense = P.ckpt > 0 ? std::min(cfg->ckpt_prefix, nt) : 0;
  P.e_min = bf.lo;
  P.e_max = bf.hi;
  P.damping = damp;
  KtGeom &g = P.g;
  g = KtGeom{};
  g.n_nodes = N;
  g.n_loc = nl;
  g.d = d;
  g.M = M;
  g.n_ctrl = nc;
  g.n_cterms = nterm;
  for (int t = 0; t < nterm; ++t) {
    g.cterm_ctrl[t] = gf.term_ctrl[t];
    g.cterm_node[t] = gf.ctrl_node[t];
  }
  g.n_lind = n_lind;
  g.n_pairs = (int)gf.pairs.size();
  g.K = K;
  g.max_jumps = (cfg->draws_per_traj - 1) / 2;   // 0: any jump is reported as KT_ERR_RECORD_FULL
  g.first_order = cfg->jump_scheme;
  g.draws = cfg->draws_per_traj;
  g.dt = dt;
  g.eps_bound = E;
  g.c_fwd = c_fwd;
  g.c_bwd = c_bwd;
  g.r = r;
  for (int i = 0; i < N; ++i) g.stride[i] = ipow(nl, N - 1 - i);
  for (int c = 0; c < nc; ++c) {
    g.ctrl_node[c] = md->ctrl_node[c];
    g.lam[c] = cfg->lambda_a[c];
  }

  // off-diagonal slot pattern of each node row (union over drift and controls, both directions)
  std::vector<std::vector<int>> cols((size_t)N * nl);
  int S = 0;
  for (int i = 0; i < N; ++i)
    for (int x = 0; x < nl; ++x) {
      std::vector<int> &cl = cols[(size_t)i * nl + x];
      for (int y = 0; y < nl; ++y) {
        if (y == x) continue;
        bool nz = at(gf.loc, i * nl * nl, nl, x, y) != 0.0 || at(gb.loc, i * nl * nl, nl, x, y) != 0.0;
        for (int t = 0; t < nterm; ++t)
          if (gf.ctrl_node[t] == i)
            nz = nz || at(gf.ctrl, t * nl * nl, nl, x, y) != 0.0 || at(gb.ctrl, t * nl * nl, nl, x, y) != 0.0;
        if (nz) cl.push_back(y);
      }
      S = std::max(S, (int)cl.size());
    }
  if (S > KT_MAX_S) return fail(KT_ERR_UNSUPPORTED, "a node row has %d > %d off-diagonal entries", S, KT_MAX_S);
  if (cfg->items_per_thread != 0 && cfg->items_per_thread != 1 && cfg->items_per_thread != 2 &&
      cfg->items_per_thread != 4 && cfg->items_per_thread != 8 && cfg->items_per_thread != 16)
    return fail(KT_ERR_ARG, "items_per_thread must be 0 (automatic), 1, 2, 4, 8 or 16");
  // automatic mapping: one thread per last-node fiber, unless a trajectory has fewer than 16 fibers
  // (d <= 81) and the tile width is automatic too (or fixed at 1 by a density matrix's single state):
  // then a CTA would hold a few warps at most, and the strided mapping with one item per thread runs
  // n_loc times as many threads per trajectory (measured faster at d = 36 and 81, about 5x in FP64,
  // where the fiber kernels' register arrays spill)
  const bool small = (nl == 6 || nl == 9) && d / nl < 16 && (cfg->tile_traj <= 0 || density);
  const int ipt = cfg->items_per_thread > 0 ? cfg->items_per_thread : (small ? 1 : 0);
  const bool fiber = (nl == 6 || nl == 9) && ipt == 0;
  const bool acs = fiber && cavity_structure(gf, gb, lo_dl, lo_val, ra_dl, ra_val);
  const bool ri = acs && S <= 2 && ri_classes(gf, gb, lo_val, ra_val, cols) && acs_constants_ok(gf, gb, lo_val, ra_val);
  if (ri) S = 2;
  g.S = std::max(S, 1);
  int SH = 1;
  for (int t = 0; t < nterm; ++t)
    for (int x = 0; x < nl; ++x) {
      int n = 0;
      for (int y = 0; y < nl; ++y) n += at(gf.ctrl, t * nl * nl, nl, x, y) != 0.0;
      SH = std::max(SH, n);
    }
  if (SH > KT_MAX_SH) return fail(KT_ERR_UNSUPPORTED, "a control factor row has %d > %d entries", SH, KT_MAX_SH);
  g.SH = SH;

  // ---- tile width, threads per CTA, items per thread
  const int esz = P.fp64 ? 16 : 8;
  const int maxthr = P.fp64 ? 512 : 1024;
  if (cfg->tile_traj > 0 && ((cfg->tile_traj & (cfg->tile_traj - 1)) || cfg->tile_traj > 32))
    return fail(KT_ERR_ARG, "tile_traj must be a power of two <= 32");
  // fiber mapping (one thread per run of n_loc elements along the last node) for the compiled
  // local dimensions; otherwise the strided mapping with 4, 8 or 16 items per thread
  const int fiber_max_threads = 736;   // the fiber kernels' launch bound
  int Tsel = 0;
  // strided mapping: items per thread above 8 spill registers, so only when nothing else fits
  const long long max_items = ((long long)d > 8LL * maxthr) ? 16LL * maxthr : 8LL * maxthr;
  for (int T = 32; T >= 1; T >>= 1) {
    if (cfg->tile_traj > 0 && T != cfg->tile_traj) continue;
    KtGeom t = g;
    t.T = T;
    if (fiber) {
      if ((long long)(d / nl) * T > fiber_max_threads) continue;
      t.nthreads = ((d / nl) * T + 31) / 32 * 32;
    } else if (ipt > 0) {
      if (((long long)d * T + ipt - 1) / ipt > maxthr) continue;
      t.nthreads = maxthr;
    } else {
      if ((long long)d * T > (cfg->tile_traj > 0 ? 16LL * maxthr : max_items)) continue;
      t.nthreads = maxthr;
    }
    if (kt_smem_bytes(t, esz, false) > 227 * 1024) continue;
    // small problems on the automatic strided mapping: tiles of at most 128 items (a few warps),
    // latency rather than throughput decides there
    if (small && cfg->items_per_thread == 0 && cfg->tile_traj <= 0 && T > 1 && (long long)d * T > 128) continue;
    Tsel = T;
    // prefer more tiles when the trajectories would not fill the GPU
    // (a shard plans with the whole problem's trajectory count: every shard needs the same tile width)
    const int Mh = sharded ? cfg->M_total : M;
    if (cfg->tile_traj <= 0 && (Mh + T - 1) / T < 2 * 152 && T > 1 && (long long)d * (T / 2) >= 256) continue;
    break;
  }
  if (Tsel == 0) return fail(KT_ERR_UNSUPPORTED, "dimension %d does not fit one trajectory tile in shared memory", d);
  g.T = Tsel;
  g.n_tiles = (M + Tsel - 1) / Tsel;
  g.M_pad = g.n_tiles * Tsel;
  g.M_norm = (double)(sharded ? cfg->M_total : M);
  g.inject_timeout = cfg->inject_copy_timeout != 0;
  if (sharded) {
    if (cfg->traj_offset % Tsel != 0 || (cfg->traj_offset + M != cfg->M_total && M % Tsel != 0))
      return fail(KT_ERR_ARG, "shard boundaries must fall on tile boundaries (tile width %d)", Tsel);
    P.sharded = 1;
    P.M_total = cfg->M_total;
    P.tile_off = cfg->traj_offset / Tsel;
    P.n_tiles_total = (cfg->M_total + Tsel - 1) / Tsel;
  }
  g.tile_elems = (d * Tsel + 3) / 4 * 4;
  {
    KtGeom t = g;
    t.nthreads = fiber ? std::max(32, ((d / nl) * Tsel + 31) / 32 * 32) : maxthr;
    const size_t smem3 = kt_smem_bytes(t, esz, true);
    g.prefetch_chi = smem3 <= 227 * 1024 ? 1 : 0;
    // backward kernel: when the tiles need several waves and a third buffer fits, CTAs loop over
    // tiles (about one CTA per SM slot) and prefetch the next tile's input during the current series
    int dev = 0, sms = 0;
    g.bwd_grid = 0;
    g.fwd_grid = 0;
    if (g.prefetch_chi && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0) {
      const int per_sm = std::max(1, std::min((int)((227 * 1024) / smem3), 2048 / std::max(32, t.nthreads)));
      if (g.n_tiles > sms * per_sm) g.bwd_grid = sms * per_sm;
      // forward kernel: the same tile loop when a fourth buffer (the next tile's psi) fits as well
      const size_t smem4 = kt_smem_bytes(t, esz, true, true);
      if (smem4 <= 227 * 1024) {
        const int per_sm4 = std::max(1, std::min((int)((227 * 1024) / smem4), 2048 / std::max(32, t.nthreads)));
        if (g.n_tiles > sms * per_sm4) g.fwd_grid = sms * per_sm4;
      }
    }
  }
  if (fiber) {
    // launcher codes -(100 v + nl): v = 0 fiber, 1 cavity structure, 2 the same with T = 1 compiled
    // in, 3 cavity structure with real / imaginary couplings, 4 the same with T = 1 (n_loc = 9)
    int v = 0;
    if (acs) v = ri ? (nl == 9 && Tsel == 1 ? 4 : 3) : (nl == 9 && Tsel == 1 ? 2 : 1);
    P.ept = -(100 * v + nl);
    g.nthreads = std::max(32, ((d / nl) * Tsel + 31) / 32 * 32);
  } else {
    const int items = d * Tsel;
    int ept = ipt > 0 ? ipt : 4;
    while ((items + ept - 1) / ept > maxthr) ept *= 2;
    P.ept = ept;
    g.nthreads = std::max(32, ((items + ept - 1) / ept + 31) / 32 * 32);
  }

  // ---- generator tables (scaled by 1/r) for both directions
  auto build_image = [&](const Gen &gen, double cgen, HostImage &im) {
    const int nls = nl * g.S;
    im.dl.assign((size_t)N * nls, 0);
    im.base.assign((size_t)N * nls, KtCplx{0, 0});
    im.cslot.assign((size_t)nterm * nls, KtCplx{0, 0});
    im.dg.assign((size_t)N * nl, KtCplx{0, 0});
    im.cdg.assign((size_t)nterm * nl, KtCplx{0, 0});
    for (int i = 0; i < N; ++i)
      for (int x = 0; x < nl; ++x) {
        const std::vector<int> &cl = cols[(size_t)i * nl + x];
        for (size_t q = 0; q < cl.size(); ++q) {
          if (cl[q] == x) continue;                  // empty slot
          const size_t e = (size_t)i * nls + x * g.S + q;
          im.dl[e] = cl[q] - x;
          const cd v = at(gen.loc, i * nl * nl, nl, x, cl[q]) / r;
          im.base[e] = KtCplx{v.real(), v.imag()};
        }
        cd dv = at(gen.loc, i * nl * nl, nl, x, x) / r;
        if (i == 0) dv -= cgen / r;
        im.dg[(size_t)i * nl + x] = KtCplx{dv.real(), dv.imag()};
      }
    for (int t = 0; t < nterm; ++t) {
      const int i = gen.ctrl_node[t];
      for (int x = 0; x < nl; ++x) {
        const std::vector<int> &cl = cols[(size_t)i * nl + x];
        for (size_t q = 0; q < cl.size(); ++q) {
          if (cl[q] == x) continue;
          const cd v = at(gen.ctrl, t * nl * nl, nl, x, cl[q]) / r;
          im.cslot[(size_t)t * nls + x * g.S + q] = KtCplx{v.real(), v.imag()};
        }
        const cd dv = at(gen.ctrl, t * nl * nl, nl, x, x) / r;
        im.cdg[(size_t)t * nl + x] = KtCplx{dv.real(), dv.imag()};
      }
    }
    const int nl2 = nl * nl;
    im.pc.assign((size_t)std::max(1, g.n_pairs), KtCplx{0, 0});
    im.poff.assign((size_t)g.n_pairs * nl2, 0);
    im.pval.assign((size_t)g.n_pairs * nl2, KtCplx{0, 0});
    for (int q = 0; q < g.n_pairs; ++q) {
      const Pair &pr = gen.pairs[q];
      im.pdst[q] = pr.dst;
      im.psrc[q] = pr.src;
      im.pc[q] = KtCplx{(pr.coef / r).real(), (pr.coef / r).imag()};
      const bool rd = pr.kind != 1, rs = pr.kind == 2;     // raise the dst / src node?
      for (int xd = 0; xd < nl; ++xd)
        for (int xs = 0; xs < nl; ++xs) {
          const cd vd = rd ? ra_val[xd] : lo_val[xd], vs = rs ? ra_val[xs] : lo_val[xs];
          if (vd == 0.0 || vs == 0.0) continue;
          const size_t e = (size_t)q * nl2 + xd * nl + xs;
          im.poff[e] = (rd ? ra_dl[xd] : lo_dl[xd]) * g.stride[pr.dst] + (rs ? ra_dl[xs] : lo_dl[xs]) * g.stride[pr.src];
          const cd v = pr.coef * vd * vs / r;
          im.pval[e] = KtCplx{v.real(), v.imag()};
        }
    }
    if (ri) {
      // constants of the real / imaginary kernels: the values the shared tables would hold
      const int last = N - 1, NP = nl / 3, NC = NP - 1;
      for (int x = 0; x < nl; ++x) {
        im.kd[2 * x] = im.dg[(size_t)last * nl + x].re;
        im.kd[2 * x + 1] = im.dg[(size_t)last * nl + x].im;
      }
      auto slot_re = [&](int x, int y) {
        for (int q = 0; q < g.S; ++q) {
          const size_t e = (size_t)last * nls + x * g.S + q;
          if (im.dl[e] == y - x) return im.base[e].re;
        }
        return 0.0;
      };
      for (int n = 1; n <= NC; ++n) {
        const int qr = 2 * NP + n - 1, qg = n;
        im.kc[n - 1] = slot_re(qr, qg);
        im.kc[NC + n - 1] = slot_re(qg, qr);
      }
      for (int q = 0; q < g.n_pairs; ++q) im.kp[q] = im.pc[q].im;
    }
    im.cf.resize(K);
    const cd ph = std::exp(cd(0.0, -cgen * dt));
    for (int k = 0; k < K; ++k) {
      const cd v = (k == 0 ? 1.0 : 2.0) * J[k] * std::pow(cd(0.0, -1.0), k) * ph;
      im.cf[k] = KtCplx{v.real(), v.imag()};
    }
  };
  build_image(gf, c_fwd, P.fwd);
  build_image(gb, c_bwd, P.bwd);

  // ---- shared operators
  P.lo_dl = lo_dl;
  P.ra_dl = ra_dl;
  P.lo_val.resize(nl);
  P.ra_val.resize(nl);
  for (int x = 0; x < nl; ++x) {
    P.lo_val[x] = KtCplx{lo_val[x].real(), lo_val[x].imag()};
    P.ra_val[x] = KtCplx{ra_val[x].real(), ra_val[x].imag()};
  }
  P.lind.assign((size_t)std::max(1, n_lind) * N, KtCplx{0, 0});
  for (int e = 0; e < n_lind * N; ++e) P.lind[e] = KtCplx{md->lind_coef[2 * e], md->lind_coef[2 * e + 1]};
  // control factors of the update overlap, one table per control term (unscaled dG/deps_c part)
  P.hc_dl.assign((size_t)nterm * nl * SH, 0);
  P.hc_val.assign((size_t)nterm * nl * SH, KtCplx{0, 0});
  for (int t = 0; t < nterm; ++t)
    for (int x = 0; x < nl; ++x) {
      int q = 0;
      for (int y = 0; y < nl; ++y) {
        const cd v = gf.ctrl[(size_t)t * nl * nl + x * nl + y];
        if (v == 0.0) continue;
        P.hc_dl[((size_t)t * nl + x) * SH + q] = y - x;
        P.hc_val[((size_t)t * nl + x) * SH + q] = KtCplx{v.real(), v.imag()};
        ++q;
      }
    }
  P.digits.resize(d);
  for (int x = 0; x < d; ++x) {
    uint32_t w = 0;
    for (int i = 0; i < N; ++i) w |= (uint32_t)((x / g.stride[i]) % nl) << (4 * i);
    P.digits[x] = w;
  }
  P.tgt.resize(d);
  for (int x = 0; x < d; ++x) P.tgt[x] = KtCplx{psi_t[x].real(), psi_t[x].imag()};
  P.density = density ? 1 : 0;
  g.density = P.density;
  if (density) {
    P.psi0.resize((size_t)2 * d);
    for (int x = 0; x < d; ++x) {
      P.psi0[2 * x] = psi_0[x].real();
      P.psi0[2 * x + 1] = psi_0[x].imag();
    }
  }
  return KT_OK;
}

kt_status upload_image(kt_problem *p, const HostImage &h, KtGenImage &im, cudaStream_t st) {
  kt_status t;
  if ((t = upload(p, (int **)&im.loc_dl, h.dl.data(), h.dl.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.loc_base, h.base.data(), h.base.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.ctrl_slot, h.cslot.data(), h.cslot.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.diag_base, h.dg.data(), h.dg.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.ctrl_diag, h.cdg.data(), h.cdg.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (int **)&im.pair_off, h.poff.data(), h.poff.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.pair_val, h.pval.data(), h.pval.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.cheb_full, h.cf.data(), h.cf.size(), st)) != KT_OK) return t;
  if ((t = upload(p, (KtCplx **)&im.pair_coef, h.pc.data(), h.pc.size(), st)) != KT_OK) return t;
  for (int q = 0; q < KT_MAX_PAIRS; ++q) {
    im.pair_dst[q] = h.pdst[q];
    im.pair_src[q] = h.psrc[q];
    im.kp32[q] = (float)h.kp[q];
    im.kp64[q] = h.kp[q];
  }
  for (int q = 0; q < 2 * KT_MAX_NL; ++q) {
    im.kd32[q] = (float)h.kd[q];
    im.kd64[q] = h.kd[q];
  }
  for (int q = 0; q < 4; ++q) {
    im.kc32[q] = (float)h.kc[q];
    im.kc64[q] = h.kc[q];
  }
  return KT_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Automatic co-state storage (ckpt_interval = -1) from the device memory still free: keep every
// co-state if they fit, else the longest prefix t_0..t_A plus checkpoints every K after it, with
// (A, K) chosen to recompute the fewest co-states (every co-state not kept is recomputed once per
// forward sweep, so the count is about nt + 1 minus the slots kept).  A reserve stays free: 2 GiB
// or 2 % of the device, and room for the forward states a gradient sweep keeps (2 sqrt(nt) + 4).
kt_status choose_storage(kt_problem *p) {
  size_t free_b = 0, total_b = 0;
  KT_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const int nt = p->nt;
  const long long reserve = std::max<long long>(2LL << 30, (long long)(total_b / 50)) +
                            (long long)(2.0 * std::sqrt((double)nt) + 4.0) * (long long)p->state_bytes;
  const long long budget = ((long long)free_b - reserve) / (long long)p->state_bytes;
  p->ckpt_auto = true;
  if (budget >= nt + 1) {
    p->ckpt = 0;
    p->ckpt_dense = nt;
    return KT_OK;
  }
  long long best = -1;
  int bestA = 0, bestK = 0;
  for (int K = 2; K <= nt; ++K) {
    if (n_ckpt_slots(nt, 0, K) + K + 1 > budget) continue;        // not even without a prefix
    int lo = 0, hi = nt - 1;                                      // largest A < nt that fits
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (n_ckpt_slots(nt, mid, K) + K + 1 <= budget) lo = mid; else hi = mid - 1;
    }
    const long long gap = nt - lo - 1, recompute = gap - gap / K;
    if (best < 0 || recompute < best) { best = recompute; bestA = lo; bestK = K; }
  }
  if (best < 0)
    return fail(KT_ERR_OOM, "automatic co-state storage: %lld state slots of %zu bytes left, too few for any "
                "checkpoint spacing", budget, p->state_bytes);
  p->ckpt = bestK;
  p->ckpt_dense = bestA;
  return KT_OK;
}

// Allocate and upload a problem for the plan P.  A probe (autotuning) keeps no co-state storage.
kt_status create_problem(const kt_model_desc *md, const kt_config *cfg, const HostPlan &P, cudaStream_t st,
                         bool probe, kt_problem **out) {
  kt_status s;
  const int nt = cfg->nt, M = cfg->M, nc = md->n_ctrl;

  kt_problem *p = new kt_problem();
  p->g = P.g;
  p->fp64 = P.fp64;
  p->ept = P.ept;
  p->cross = P.cross;
  p->density = P.density;
  p->sharded = P.sharded;
  p->tile_off = P.tile_off;
  p->n_tiles_total = P.n_tiles_total;
  p->M_total = P.M_total;
  p->esz = P.fp64 ? 16 : 8;
  p->nt = nt;
  p->M = M;
  p->T = cfg->T;
  p->n_passes = cfg->n_passes;
  p->n_passes_alloc = cfg->n_passes;
  p->ckpt = P.ckpt;
  p->ckpt_dense = P.ckpt_dense;
  if (p->ckpt > 0 && p->ckpt_dense >= nt) p->ckpt = p->ckpt_dense = 0;   // the prefix keeps everything
  p->e_min = P.e_min;
  p->e_max = P.e_max;
  p->damping = P.damping;
  const KtGeom &g = p->g;
  p->state_bytes = (size_t)g.n_tiles * g.tile_elems * p->esz;

#define TRY(x) do { s = (x); if (s != KT_OK) { krotov_free(p); return s; } } while (0)
  TRY(upload_image(p, P.fwd, p->im_fwd, st));
  TRY(upload_image(p, P.bwd, p->im_bwd, st));
  KtOps &o = p->ops;
  TRY(upload(p, (int **)&o.lo_dl, P.lo_dl.data(), P.lo_dl.size(), st));
  TRY(upload(p, (KtCplx **)&o.lo_val, P.lo_val.data(), P.lo_val.size(), st));
  TRY(upload(p, (int **)&o.ra_dl, P.ra_dl.data(), P.ra_dl.size(), st));
  TRY(upload(p, (KtCplx **)&o.ra_val, P.ra_val.data(), P.ra_val.size(), st));
  TRY(upload(p, (KtCplx **)&o.lind_coef, P.lind.data(), P.lind.size(), st));
  TRY(upload(p, (int **)&o.hc_dl, P.hc_dl.data(), P.hc_dl.size(), st));
  TRY(upload(p, (KtCplx **)&o.hc_val, P.hc_val.data(), P.hc_val.size(), st));
  TRY(upload(p, (uint32_t **)&o.digits, P.digits.data(), P.digits.size(), st));
  TRY(upload(p, (KtCplx **)&o.tgt, P.tgt.data(), P.tgt.size(), st));

  // ---- pulses, uniforms, states, records
  TRY(upload(p, &p->eps_old, cfg->eps_guess, (size_t)nc * nt, st));
  TRY(upload(p, &p->eps_new, cfg->eps_guess, (size_t)nc * nt, st));
  std::vector<double> zeros((size_t)nc * nt, 0.0);
  TRY(upload(p, &p->deps, zeros.data(), zeros.size(), st));
  TRY(upload(p, &p->shape, cfg->shape, (size_t)nc * nt, st));
  TRY(upload(p, &p->U, cfg->uniforms, (size_t)cfg->n_passes * M * cfg->draws_per_traj, st));
  {
    std::vector<double> buf64;
    std::vector<float> buf32;
    const bool batch = !P.density && md->psi0_batch != nullptr;
    const double *src = P.density ? P.psi0.data() : (batch ? md->psi0_batch : md->psi0);
    if (p->fp64) {
      to_tiles<double>(p, src, batch, buf64);
      TRY(upload(p, (double **)&p->psi_init, buf64.data(), buf64.size(), st));
    } else {
      to_tiles<float>(p, src, batch, buf32);
      TRY(upload(p, (float **)&p->psi_init, buf32.data(), buf32.size(), st));
    }
  }
  TRY(dev_alloc(p, &p->psi[0], p->state_bytes));
  TRY(dev_alloc(p, &p->psi[1], p->state_bytes));
  const size_t Mp = g.M_pad, mj = g.max_jumps;
  TRY(dev_alloc(p, (void **)&p->rstate, Mp * sizeof(double)));
  for (int b = 0; b < 2; ++b) {
    TRY(dev_alloc(p, (void **)&p->jcount[b], Mp * sizeof(int)));
    TRY(dev_alloc(p, (void **)&p->rec_step[b], Mp * mj * sizeof(int)));
    TRY(dev_alloc(p, (void **)&p->rec_ch[b], Mp * mj * sizeof(int)));
    TRY(dev_alloc(p, (void **)&p->rec_s[b], Mp * mj * sizeof(double)));
    TRY(dev_alloc(p, (void **)&p->rec_c[b], Mp * mj * sizeof(double)));
    if (cudaMemsetAsync(p->jcount[b], 0, Mp * sizeof(int), st) != cudaSuccess) { krotov_free(p); return fail(KT_ERR_CUDA, "memset"); }
  }
  TRY(dev_alloc(p, (void **)&p->cursor, Mp * sizeof(int)));
  // two sets: a whole-sweep launch alternates them by interval parity
  TRY(dev_alloc(p, (void **)&p->partials, (size_t)2 * g.n_tiles * nc * sizeof(double)));
  if (p->sharded) {
    TRY(dev_alloc(p, (void **)&p->spart, (size_t)p->n_tiles_total * nc * sizeof(double)));
    TRY(dev_alloc(p, (void **)&p->tau_all, (size_t)p->M_total * sizeof(KtCplx)));
  }
  TRY(dev_alloc(p, (void **)&p->counter, sizeof(unsigned)));
  TRY(dev_alloc(p, (void **)&p->tau, Mp * sizeof(KtCplx)));
  TRY(dev_alloc(p, (void **)&p->norm2, Mp * sizeof(double)));
  TRY(dev_alloc(p, (void **)&p->status, sizeof(int)));
  TRY(dev_alloc(p, (void **)&p->pass, 3 * sizeof(int)));
  if (p->cross && !probe) {
    TRY(dev_alloc(p, &p->cwork, kt_cross_work_bytes(g, (int)p->esz)));
    TRY(dev_alloc(p, (void **)&p->cpart, kt_cross_partials(g) * sizeof(double)));
    TRY(dev_alloc(p, (void **)&p->cpair, kt_cross_pair_bytes(g)));
    TRY(dev_alloc(p, (void **)&p->ccounter, sizeof(unsigned)));
    if (cudaMemsetAsync(p->ccounter, 0, sizeof(unsigned), st) != cudaSuccess) {
      krotov_free(p);
      return fail(KT_ERR_CUDA, "memset failed");
    }
  }
  if (!probe) {
    // co-state storage, allocated last so that an automatic choice sees the memory left
    if (cfg->ckpt_interval == -1) TRY(choose_storage(p));
    p->n_chi_slots = n_ckpt_slots(nt, p->ckpt_dense, p->ckpt);
    TRY(dev_alloc(p, &p->chi, p->state_bytes * p->n_chi_slots));
    if (p->ckpt > 0) TRY(dev_alloc(p, &p->seg, p->state_bytes * (p->ckpt + 1)));
    // whole-sweep launches: the strided mapping (the small problems' mapping; the sweep kernels are
    // compiled for it only), every tile resident at once (the forward sweep's grid barrier), every
    // co-state kept (each interval's co-state has its slot), no exchange with other shards and no
    // pair sums between intervals
    int dev = 0, sms = 0, per = 0;
    if (!cfg->per_interval_launches && p->ept > 0 && p->ckpt == 0 && !p->sharded && !p->cross &&
        cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        kt_fwd_blocks_per_sm(p->fp64, p->ept, g, &per) == cudaSuccess && (long long)per * sms >= g.n_tiles) {
      TRY(dev_alloc(p, (void **)&p->sync, 2 * sizeof(unsigned)));
      p->whole_sweep = 1;
    }
    cudaGetLastError();   // an occupancy query that failed leaves per-interval launches
  }
  p->eps_base = p->eps_old;
  if (kt_launch_pass_reset(p->pass, p->n_passes, st) != cudaSuccess ||
      cudaMemsetAsync(p->counter, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(p->status, 0, sizeof(int), st) != cudaSuccess) {
    krotov_free(p);
    return fail(KT_ERR_CUDA, "memset failed");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    krotov_free(p);
    return fail(KT_ERR_CUDA, "initial upload failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
#undef TRY
  p->shape_h.assign(cfg->shape, cfg->shape + (size_t)nc * nt);
  p->lam_h.assign(cfg->lambda_a, cfg->lambda_a + nc);
  *out = p;
  return KT_OK;
}

// Average duration of a forward plus a backward interval kernel of probe q (no update, guess pulse,
// no jump records), timed with events on st over a few intervals after two warm-up intervals.
kt_status probe_forward_ms(kt_problem *q, cudaStream_t st, double *ms_out) {
  const int warm = 2, timed = 12;
  KT_CUDA(kt_launch_init_pass(q->g, q->U, q->pass, q->rstate, q->jcount[0], st));
  // the backward kernel follows the (empty) records of the other buffer: seek its cursor first
  KT_CUDA(kt_launch_cursor_seek(q->g, q->rec_step[1 - q->cur], q->jcount[1 - q->cur], q->nt, q->cursor, st));
  FwdArgs a = fwd_args(q, 0);
  a.chi_t = nullptr;
  BwdArgs b = bwd_args(q);
  cudaEvent_t e[2];
  KT_CUDA(cudaEventCreate(&e[0]));
  if (cudaEventCreate(&e[1]) != cudaSuccess) {
    cudaEventDestroy(e[0]);
    return fail(KT_ERR_CUDA, "cudaEventCreate failed");
  }
  cudaError_t err = cudaSuccess;
  for (int i = 0; i < warm + timed && err == cudaSuccess; ++i) {
    if (i == warm) err = cudaEventRecord(e[0], st);
    a.j = 1 + i % q->nt;
    a.psi_in = i == 0 ? q->psi_init : q->psi[(i - 1) & 1];
    a.psi_out = q->psi[i & 1];
    if (err == cudaSuccess) err = kt_launch_fwd(q->fp64, q->ept, q->g, q->im_fwd, q->ops, a, st);
    // one backward interval on the state just written (free propagation: no records)
    b.j = q->nt - i % q->nt;
    b.chi_in = q->psi[i & 1];
    b.chi_out = q->psi[(i - 1) & 1];
    if (err == cudaSuccess && i > 0) err = kt_launch_bwd(q->fp64, q->ept, q->g, q->im_bwd, q->ops, b, st);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e[1], st);
  if (err == cudaSuccess) err = cudaEventSynchronize(e[1]);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e[0], e[1]);
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  if (err != cudaSuccess) return fail(KT_ERR_CUDA, "autotuning launch failed: %s", cudaGetErrorString(err));
  *ms_out = ms / timed;
  return KT_OK;
}

// Autotuner: plan every power-of-two tile width that fits, with the automatic thread mapping and
// (unless the caller fixed items_per_thread) the strided mapping at 1, 2 and 4 items per thread,
// time a forward and a backward interval kernel of each distinct plan, keep the fastest.
kt_status autotune(const kt_model_desc *md, const kt_config *cfg, cudaStream_t st, HostPlan &best) {
  double best_ms = 0.0;
  int best_T = 0;
  kt_status last = KT_ERR_UNSUPPORTED;
  std::vector<std::pair<int, int>> seen;   // (tile width, launcher code) already timed
  const int ipts[4] = {0, 1, 2, 4};
  for (int T = 1; T <= 32; T <<= 1)
  for (int m = 0; m < (cfg->items_per_thread > 0 ? 1 : 4); ++m) {
    kt_config c = *cfg;
    c.tile_traj = T;
    if (cfg->items_per_thread == 0) c.items_per_thread = ipts[m];
    HostPlan P;
    kt_status s = plan(md, &c, P);
    if (s != KT_OK) {
      if (s != KT_ERR_UNSUPPORTED) return s;       // a descriptor error, the same for every width
      last = s;
      continue;
    }
    if (std::find(seen.begin(), seen.end(), std::make_pair(P.g.T, P.ept)) != seen.end()) continue;
    seen.emplace_back(P.g.T, P.ept);
    kt_problem *q = nullptr;
    if ((s = create_problem(md, &c, P, st, true, &q)) != KT_OK) return s;
    double ms = 0.0;
    s = probe_forward_ms(q, st, &ms);
    krotov_free(q);
    if (s != KT_OK) return s;
    if (best_T == 0 || ms < best_ms) {
      best_ms = ms;
      best_T = T;
      best = P;
    }
  }
  if (best_T == 0) return last == KT_OK ? fail(KT_ERR_UNSUPPORTED, "no tile width fits") : last;
  return KT_OK;
}

}  // namespace

// Configuration of a density-matrix problem: one Liouville-space "trajectory" whose threshold
// r = -1 can never be reached (the density matrix has no jumps), the update of Eq. krotovupdate.
static const double kNoJump = -1.0;
static kt_config density_config(const kt_config *cfg) {
  kt_config c = *cfg;
  c.M = 1;
  c.tile_traj = 1;                 // one state: one tile of width 1
  c.uniforms = &kNoJump;
  c.n_passes = 1;
  c.draws_per_traj = 1;
  c.update_rule = 0;
  c.jump_scheme = 0;
  return c;
}

extern "C" {

KT_API kt_status krotov_init_density(const kt_model_desc *md, const kt_config *cfg, void *stream, kt_problem **out) {
  if (!md || !cfg || !out) return fail(KT_ERR_ARG, "NULL descriptor or output pointer");
  *out = nullptr;
  if (cfg->tile_traj == -1) return fail(KT_ERR_ARG, "a density-matrix problem has one state: nothing to autotune");
  const kt_config c = density_config(cfg);
  HostPlan P;
  kt_status s = plan(md, &c, P, true);
  if (s != KT_OK) return s;
  return create_problem(md, &c, P, (cudaStream_t)stream, false, out);
}

KT_API kt_status krotov_init(const kt_model_desc *md, const kt_config *cfg, void *stream, kt_problem **out) {
  if (!md || !cfg || !out) return fail(KT_ERR_ARG, "NULL descriptor or output pointer");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  HostPlan P;
  kt_status s = cfg->tile_traj == -1 ? autotune(md, cfg, st, P) : plan(md, cfg, P);
  if (s != KT_OK) return s;
  return create_problem(md, cfg, P, st, false, out);
}

// Host-only expansion of the generator tables into a dense matrix, indexed exactly the way the
// kernels index them (digits, slot offsets, pair tables, diagonal), with a bounds check on every
// neighbour.  direction 0: G = H_eff(eps); direction 1: G = -H_eff(eps)^dag.  out [d][d][2].
KT_API kt_status kt_generator_dense(const kt_model_desc *md, const kt_config *cfg, int direction, const double *eps,
                                    double *out) {
  if (!out || !eps) return fail(KT_ERR_ARG, "NULL argument");
  if (direction < 0 || direction > 3) return fail(KT_ERR_ARG, "direction must be 0..3");
  HostPlan P;
  kt_status s;
  if (direction >= 2) {
    kt_config c = density_config(cfg);
    s = plan(md, &c, P, true);
  } else {
    s = plan(md, cfg, P);
  }
  if (s != KT_OK) return s;
  const KtGeom &g = P.g;
  const HostImage &im = (direction & 1) ? P.bwd : P.fwd;
  const double cgen = (direction & 1) ? g.c_bwd : g.c_fwd;
  const int d = g.d, nl = g.n_loc, nls = nl * g.S, nl2 = nl * nl;
  std::fill(out, out + (size_t)d * d * 2, 0.0);
  auto add = [&](int x, int y, cd v) -> bool {
    if (y < 0 || y >= d) return false;
    out[((size_t)x * d + y) * 2] += v.real();
    out[((size_t)x * d + y) * 2 + 1] += v.imag();
    return true;
  };
  for (int x = 0; x < d; ++x) {
    const uint32_t dig = P.digits[x];
    cd dv = 0.0;
    for (int i = 0; i < g.n_nodes; ++i) {
      const int xi = (dig >> (4 * i)) & 15;
      dv += cd(im.dg[(size_t)i * nl + xi].re, im.dg[(size_t)i * nl + xi].im);
      for (int t = 0; t < g.n_cterms; ++t)
        if (g.cterm_node[t] == i)
          dv += eps[g.cterm_ctrl[t]] * cd(im.cdg[(size_t)t * nl + xi].re, im.cdg[(size_t)t * nl + xi].im);
      for (int q = 0; q < g.S; ++q) {
        const size_t e = (size_t)i * nls + xi * g.S + q;
        if (!im.dl[e]) continue;
        cd v(im.base[e].re, im.base[e].im);
        for (int t = 0; t < g.n_cterms; ++t)
          if (g.cterm_node[t] == i)
            v += eps[g.cterm_ctrl[t]] * cd(im.cslot[(size_t)t * nls + xi * g.S + q].re, im.cslot[(size_t)t * nls + xi * g.S + q].im);
        if (!add(x, x + im.dl[e] * g.stride[i], v * g.r)) return fail(KT_ERR_RANGE, "node entry leaves the space at row %d", x);
      }
    }
    for (int q = 0; q < g.n_pairs; ++q) {
      const int xd = (dig >> (4 * im.pdst[q])) & 15, xs = (dig >> (4 * im.psrc[q])) & 15;
      const size_t e = (size_t)q * nl2 + xd * nl + xs;
      if (!im.poff[e]) continue;
      if (!add(x, x + im.poff[e], cd(im.pval[e].re, im.pval[e].im) * g.r))
        return fail(KT_ERR_RANGE, "pair entry leaves the space at row %d", x);
    }
    add(x, x, dv * g.r + cgen);
  }
  return KT_OK;
}

KT_API kt_status propagate_forward(kt_problem *p, int sequential_update, double *F_out, void *stream) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  cudaStream_t st = (cudaStream_t)stream;
  if (sequential_update < 0 || sequential_update > 2) return fail(KT_ERR_ARG, "sequential_update must be 0, 1 or 2");
  kt_status s;
  if (sequential_update == 2 && (s = grad_setup(p, st)) != KT_OK) return s;
  s = forward_sweep(p, sequential_update == 1 ? 1 : 0, st, sequential_update == 2);
  if (s != KT_OK) return s;
  if (F_out) return host_fidelity(p, F_out, nullptr, st);
  return KT_OK;
}

KT_API kt_status propagate_backward(kt_problem *p, void *stream) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  return backward_sweep(p, (cudaStream_t)stream);
}

KT_API kt_status krotov_update(kt_problem *p, int n_iter, double *JT_out, double *J_out, void *stream) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  if (n_iter < 0) return fail(KT_ERR_ARG, "n_iter < 0");
  cudaStream_t st = (cudaStream_t)stream;
  kt_status s;
  if (!p->have_fwd && (s = forward_sweep(p, 0, st)) != KT_OK) return s;
  std::vector<double> de;
  for (int it = 0; it < n_iter; ++it) {
    if (p->profiling) {
      // per-launch event pairs need the launches issued one by one
      if ((s = backward_sweep(p, st)) != KT_OK) return s;
      if ((s = forward_sweep(p, 1, st)) != KT_OK) return s;
    } else if ((s = graph_iteration(p, st)) != KT_OK) {
      return s;
    }
    if (JT_out || J_out) {
      double F = 0.0;
      if ((s = host_fidelity(p, &F, nullptr, st)) != KT_OK) return s;
      if (JT_out) JT_out[it] = 1.0 - F;
      if (J_out) {
        de.resize((size_t)p->g.n_ctrl * p->nt);
        KT_CUDA(cudaMemcpyAsync(de.data(), p->deps, de.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        KT_CUDA(cudaStreamSynchronize(st));
        double J = 1.0 - F;
        for (int c = 0; c < p->g.n_ctrl; ++c)
          for (int j = 0; j < p->nt; ++j) {
            const double S = p->shape_h[(size_t)c * p->nt + j];
            if (S > 0.0) J += p->lam_h[c] * de[(size_t)c * p->nt + j] * de[(size_t)c * p->nt + j] * p->g.dt / S;
          }
        J_out[it] = J;
      }
    }
  }
  return KT_OK;
}

KT_API kt_status fidelity(kt_problem *p, double *F_out, double *tau_out) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  if (!p->have_fwd) return fail(KT_ERR_STATE, "no forward sweep yet");
  return host_fidelity(p, F_out, tau_out, 0);
}

KT_API kt_status krotov_get_pulses(kt_problem *p, double *eps_out) {
  if (!p || !eps_out) return fail(KT_ERR_ARG, "NULL argument");
  KT_CUDA(cudaMemcpy(eps_out, p->eps_old, sizeof(double) * p->g.n_ctrl * p->nt, cudaMemcpyDeviceToHost));
  return KT_OK;
}

KT_API kt_status krotov_get_update(kt_problem *p, double *deps_out) {
  if (!p || !deps_out) return fail(KT_ERR_ARG, "NULL argument");
  KT_CUDA(cudaMemcpy(deps_out, p->deps, sizeof(double) * p->g.n_ctrl * p->nt, cudaMemcpyDeviceToHost));
  return KT_OK;
}

KT_API kt_status krotov_set_pulses(kt_problem *p, const double *eps) {
  if (!p || !eps) return fail(KT_ERR_ARG, "NULL argument");
  const size_t n = (size_t)p->g.n_ctrl * p->nt;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(eps[i]) || std::fabs(eps[i]) > p->g.eps_bound)
      return fail(KT_ERR_RANGE, "pulse value %zu non-finite or beyond eps_bound", i);
  KT_CUDA(cudaMemcpy(p->eps_old, eps, n * sizeof(double), cudaMemcpyHostToDevice));
  KT_CUDA(cudaMemcpy(p->eps_new, eps, n * sizeof(double), cudaMemcpyHostToDevice));
  p->have_fwd = p->have_bwd = false;
  p->grad_ready = false;
  return KT_OK;
}

KT_API kt_status krotov_get_records(kt_problem *p, int *count_out, int *step_out, int *channel_out, double *s_out,
                                    double *c_out) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  if (!p->have_fwd) return fail(KT_ERR_STATE, "no forward sweep yet");
  const int prev = 1 - p->cur;
  const size_t M = p->M, mj = p->g.max_jumps;
  if (count_out) KT_CUDA(cudaMemcpy(count_out, p->jcount[prev], M * sizeof(int), cudaMemcpyDeviceToHost));
  if (step_out) KT_CUDA(cudaMemcpy(step_out, p->rec_step[prev], M * mj * sizeof(int), cudaMemcpyDeviceToHost));
  if (channel_out) KT_CUDA(cudaMemcpy(channel_out, p->rec_ch[prev], M * mj * sizeof(int), cudaMemcpyDeviceToHost));
  if (s_out) KT_CUDA(cudaMemcpy(s_out, p->rec_s[prev], M * mj * sizeof(double), cudaMemcpyDeviceToHost));
  if (c_out) KT_CUDA(cudaMemcpy(c_out, p->rec_c[prev], M * mj * sizeof(double), cudaMemcpyDeviceToHost));
  return KT_OK;
}

KT_API kt_status krotov_get_states(kt_problem *p, double *psi_out) {
  if (!p || !psi_out) return fail(KT_ERR_ARG, "NULL argument");
  if (!p->have_fwd) return fail(KT_ERR_STATE, "no forward sweep yet");
  return download_state(p, p->psi[p->final_buf], psi_out, 0);
}

KT_API kt_status krotov_get_costate(kt_problem *p, int j, double *chi_out) {
  if (!p || !chi_out) return fail(KT_ERR_ARG, "NULL argument");
  if (!p->have_bwd) return fail(KT_ERR_STATE, "no backward sweep since the last forward sweep");
  if (j < 0 || j > p->nt || !is_ckpt(p, j)) return fail(KT_ERR_ARG, "co-state %d not stored", j);
  return download_state(p, ckpt_slot(p, j), chi_out, 0);
}

KT_API kt_status krotov_set_pulses_device(kt_problem *p, const double *eps_dev, void *stream) {
  if (!p || !eps_dev) return fail(KT_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)p->g.n_ctrl * p->nt;
  KT_CUDA(cudaMemcpyAsync(p->eps_old, eps_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KT_CUDA(cudaMemcpyAsync(p->eps_new, eps_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  KT_CUDA(kt_launch_pulse_check(p->eps_old, (long long)n, p->g.eps_bound, p->status, st));
  p->have_fwd = p->have_bwd = false;
  p->grad_ready = false;
  return KT_OK;
}

KT_API kt_status krotov_gradient(kt_problem *p, const double *eps_dev, double *dJ_dev, void *stream) {
  if (!p || !dJ_dev) return fail(KT_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  kt_status s;
  if (eps_dev) {
    if ((s = krotov_set_pulses_device(p, eps_dev, stream)) != KT_OK) return s;
    if ((s = grad_setup(p, st)) != KT_OK) return s;
    if ((s = forward_sweep(p, 0, st, true)) != KT_OK) return s;
  }
  if ((s = gradient_sweep(p, st)) != KT_OK) return s;
  KT_CUDA(cudaMemcpyAsync(dJ_dev, p->dgrad, sizeof(double) * p->g.n_ctrl * p->nt, cudaMemcpyDeviceToDevice, st));
  return KT_OK;
}

KT_API kt_status krotov_get_JT(kt_problem *p, double *JT_dev, void *stream) {
  if (!p || !JT_dev) return fail(KT_ERR_ARG, "NULL argument");
  if (!p->have_fwd) return fail(KT_ERR_STATE, "no forward sweep yet");
  KT_CUDA(kt_launch_functional(p->tau, p->M, p->density, JT_dev, (cudaStream_t)stream));
  return KT_OK;
}

KT_API kt_status krotov_pulse_noise(kt_problem *p, const double *ref, double *nu_out, void *stream) {
  if (!p || !nu_out) return fail(KT_ERR_ARG, "NULL argument");
  if (p->nt < 5) return fail(KT_ERR_ARG, "the five-point smoothing needs nt >= 5");
  cudaStream_t st = (cudaStream_t)stream;
  const int nc = p->g.n_ctrl;
  const size_t n = (size_t)nc * p->nt;
  if (!p->nu) {
    kt_status s = dev_alloc(p, (void **)&p->nu, KT_MAX_CTRL * sizeof(double));
    if (s == KT_OK) s = dev_alloc(p, (void **)&p->nu_ref, n * sizeof(double));
    if (s != KT_OK) return s;
  }
  if (ref) KT_CUDA(cudaMemcpyAsync(p->nu_ref, ref, n * sizeof(double), cudaMemcpyHostToDevice, st));
  KT_CUDA(kt_launch_pulse_noise(p->eps_old, ref ? p->nu_ref : nullptr, nc, p->nt, p->g.dt, p->nu, st));
  KT_CUDA(cudaMemcpyAsync(nu_out, p->nu, nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  KT_CUDA(cudaStreamSynchronize(st));
  return KT_OK;
}

KT_API kt_status krotov_set_uniforms(kt_problem *p, const double *uniforms, int n_passes, void *stream) {
  if (!p || !uniforms) return fail(KT_ERR_ARG, "NULL argument");
  if (n_passes < 1 || n_passes > p->n_passes_alloc)
    return fail(KT_ERR_ARG, "n_passes must be in [1, %d] (the value given at init)", p->n_passes_alloc);
  const size_t n = (size_t)n_passes * p->M * p->g.draws;
  cudaStream_t st = (cudaStream_t)stream;
  KT_CUDA(cudaMemcpyAsync(p->U, uniforms, n * sizeof(double), cudaMemcpyDefault, st));   // host or device memory
  KT_CUDA(kt_launch_pass_reset(p->pass, n_passes, st));
  p->n_passes = n_passes;
  p->passes = 0;
  return KT_OK;
}

KT_API kt_status krotov_set_profiling(kt_problem *p, int on) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  p->profiling = on != 0;
  p->ev_used = 0;
  for (int f = 0; f < KT_PROF_FAMILIES; ++f) {
    p->prof_ms[f] = 0.0;
    p->prof_launches[f] = 0;
  }
  return KT_OK;
}

KT_API kt_status krotov_get_profile(kt_problem *p, double *ms_out, long long *launches_out) {
  if (!p) return fail(KT_ERR_ARG, "NULL problem");
  for (int f = 0; f < KT_PROF_FAMILIES; ++f) {
    if (ms_out) ms_out[f] = p->prof_ms[f];
    if (launches_out) launches_out[f] = p->prof_launches[f];
  }
  return KT_OK;
}

KT_API kt_status krotov_get_info(kt_problem *p, kt_info *info) {
  if (!p || !info) return fail(KT_ERR_ARG, "NULL argument");
  info->d = p->g.d;
  info->max_jumps = p->g.max_jumps;
  info->cheb_terms = p->g.K;
  info->tile_traj = p->g.T;
  info->n_tiles = p->g.n_tiles;
  info->threads = p->g.nthreads;
  info->e_min = p->e_min;
  info->e_max = p->e_max;
  info->damping = p->damping;
  info->device_bytes = (long long)p->bytes;
  info->passes = p->passes;
  info->eps_bound = p->g.eps_bound;
  info->sweeps = p->sweeps;
  info->ckpt_interval = p->ckpt;
  info->ckpt_kept_prefix = p->ckpt == 0 ? p->nt : p->ckpt_dense;
  info->costate_slots = p->n_chi_slots;
  info->items_per_thread = p->ept > 0 ? p->ept : 0;
  info->whole_sweep = p->whole_sweep;
  return KT_OK;
}

}  // extern "C"

// ============================================================================ batches of problems
// Independent problems (their own model, size, precision and buffers) whose Krotov iterations
// run as one CUDA graph launch: each problem's captured iteration is a child graph of the batch
// graph, with no edges between problems, so the device schedules their interval kernels
// concurrently.
struct kt_batch {
  std::vector<kt_problem *> probs;
  struct Entry {
    std::vector<int> keys;      // iter_key of every problem the graph was built for
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long nodes = 0;
  };
  Entry cache[2];               // the two buffer states an iteration alternates between
  int next_slot = 0;
};

namespace {

void drop_entry(kt_batch::Entry &e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  e = kt_batch::Entry{};
}

kt_status batch_graph(kt_batch *b, kt_batch::Entry **out) {
  std::vector<int> keys(b->probs.size());
  for (size_t i = 0; i < b->probs.size(); ++i) keys[i] = iter_key(b->probs[i]);
  for (kt_batch::Entry &e : b->cache)
    if (e.exec && e.keys == keys) {
      *out = &e;
      return KT_OK;
    }
  kt_batch::Entry &e = b->cache[b->next_slot];
  b->next_slot ^= 1;
  drop_entry(e);
  KT_CUDA(cudaGraphCreate(&e.graph, 0));
  for (size_t i = 0; i < b->probs.size(); ++i) {
    cudaGraph_t child;
    kt_status s = capture_iteration(b->probs[i], &child);
    if (s != KT_OK) {
      drop_entry(e);
      return s;
    }
    size_t n = 0;
    cudaGraphNode_t node;
    if (cudaGraphGetNodes(child, nullptr, &n) != cudaSuccess ||
        cudaGraphAddChildGraphNode(&node, e.graph, nullptr, 0, child) != cudaSuccess) {
      drop_entry(e);
      return fail(KT_ERR_CUDA, "building the batch graph failed at problem %zu", i);
    }
    e.nodes += (long long)n;
  }
  const cudaError_t err = cudaGraphInstantiate(&e.exec, e.graph, 0);
  if (err != cudaSuccess) {
    drop_entry(e);
    return fail(KT_ERR_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(err));
  }
  e.keys = keys;
  *out = &e;
  return KT_OK;
}

// Prefix the calling thread's last error with the problem index.
kt_status batch_fail(kt_status s, size_t i) {
  const std::string msg = g_err;
  return fail(s, "problem %zu: %s", i, msg.c_str());
}

}  // namespace

extern "C" {

KT_API kt_status krotov_init_batch(const kt_model_desc *const *models, const kt_config *const *cfgs, int n,
                                   void *stream, kt_batch **out) {
  if (!models || !cfgs || !out) return fail(KT_ERR_ARG, "NULL descriptor array or output pointer");
  *out = nullptr;
  if (n < 1) return fail(KT_ERR_ARG, "a batch needs n >= 1 problems");
  kt_batch *b = new kt_batch();
  for (int i = 0; i < n; ++i) {
    kt_problem *p = nullptr;
    const kt_status s = krotov_init(models[i], cfgs[i], stream, &p);
    if (s != KT_OK) {
      krotov_batch_free(b);
      return batch_fail(s, (size_t)i);
    }
    // the problems of a batch run side by side in one graph: per-interval launches, so that no
    // cooperative launch has to wait for the SMs the other problems hold
    p->whole_sweep = 0;
    b->probs.push_back(p);
  }
  *out = b;
  return KT_OK;
}

KT_API kt_status krotov_batch_update(kt_batch *b, int n_iter, double *JT_out, void *stream) {
  if (!b) return fail(KT_ERR_ARG, "NULL batch");
  if (n_iter < 0) return fail(KT_ERR_ARG, "n_iter < 0");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = b->probs.size();
  kt_status s;
  // guess sweeps, on the problems' own streams so that they overlap
  {
    cudaEvent_t ready;
    KT_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ready, st);
    std::vector<size_t> started;
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
      kt_problem *p = b->probs[i];
      if (p->have_fwd) continue;
      if (!p->cap_stream) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->cap_stream, ready, 0);
      if (e != cudaSuccess) break;
      if ((s = enqueue_forward(p, 0, p->cap_stream, false)) != KT_OK) {
        cudaEventDestroy(ready);
        return batch_fail(s, i);
      }
      started.push_back(i);
    }
    cudaEventDestroy(ready);
    if (e != cudaSuccess) return fail(KT_ERR_CUDA, "guess sweeps: %s", cudaGetErrorString(e));
    for (size_t i : started) {
      if ((s = read_status(b->probs[i], b->probs[i]->cap_stream)) != KT_OK) return batch_fail(s, i);
      commit_forward(b->probs[i], 0, false);
    }
  }
  for (int it = 0; it < n_iter; ++it) {
    kt_batch::Entry *e = nullptr;
    if ((s = batch_graph(b, &e)) != KT_OK) return s;
    KT_CUDA(cudaGraphLaunch(e->exec, st));
    kt_status first = KT_OK;
    size_t first_i = 0;
    for (size_t i = 0; i < n; ++i) {
      kt_problem *p = b->probs[i];
      s = read_status(p, st);
      if (s != KT_OK) {
        if (first == KT_OK) {
          first = s;
          first_i = i;
        }
        p->have_fwd = p->have_bwd = false;
        continue;
      }
      commit_iteration(p);
    }
    if (first != KT_OK) return batch_fail(first, first_i);
    if (JT_out)
      for (size_t i = 0; i < n; ++i) {
        double F = 0.0;
        if ((s = host_fidelity(b->probs[i], &F, nullptr, st)) != KT_OK) return batch_fail(s, i);
        JT_out[(size_t)it * n + i] = 1.0 - F;
      }
  }
  return KT_OK;
}

KT_API kt_status krotov_batch_problem(kt_batch *b, int i, kt_problem **out) {
  if (!b || !out) return fail(KT_ERR_ARG, "NULL argument");
  if (i < 0 || i >= (int)b->probs.size()) return fail(KT_ERR_ARG, "problem index %d out of range", i);
  *out = b->probs[i];
  return KT_OK;
}

KT_API kt_status krotov_batch_info(kt_batch *b, int *n_problems, long long *graph_nodes, long long *device_bytes) {
  if (!b) return fail(KT_ERR_ARG, "NULL batch");
  if (n_problems) *n_problems = (int)b->probs.size();
  if (graph_nodes) {
    *graph_nodes = 0;
    for (const kt_batch::Entry &e : b->cache) *graph_nodes = std::max(*graph_nodes, e.nodes);
  }
  if (device_bytes) {
    long long t = 0;
    for (const kt_problem *p : b->probs) t += (long long)p->bytes;
    *device_bytes = t;
  }
  return KT_OK;
}

KT_API void krotov_batch_free(kt_batch *b) {
  if (!b) return;
  for (kt_batch::Entry &e : b->cache) drop_entry(e);
  for (kt_problem *p : b->probs) krotov_free(p);
  delete b;
}

}  // extern "C"

// ============================================================================ trajectory sharding
// A problem's trajectories split into shards (kt_config.traj_offset / M_total): every shard
// propagates its own trajectories, and the only exchange is, once per interval, the per-tile partial
// sums of the update overlap (Sec. 2.3: the trajectories are independent, only scalars are
// communicated), after which every shard forms the same Delta eps in the single-GPU order.
struct kt_group {
  std::vector<kt_problem *> shards;   // borrowed, ordered by trajectory offset
};

namespace {

// Forward sweep of every shard of a group, interval by interval on one stream: the shards' overlaps at
// t_j, the partial slices copied into every shard's copy of the global array, then Delta eps.
kt_status group_forward(kt_group *gr, int update, cudaStream_t st) {
  const size_t n = gr->shards.size();
  std::vector<FwdArgs> a(n);
  kt_status s;
  for (size_t i = 0; i < n; ++i)
    if ((s = fwd_begin(gr->shards[i], update, st, a[i])) != KT_OK) return s;
  const int nt = gr->shards[0]->nt;
  auto exchange = [&](int j) -> kt_status {
    for (kt_problem *src : gr->shards) {
      const size_t off = (size_t)src->tile_off * src->g.n_ctrl, len = (size_t)src->g.n_tiles * src->g.n_ctrl;
      for (kt_problem *dst : gr->shards)
        if (dst != src)
          KT_CUDA(cudaMemcpyAsync(dst->spart + off, src->spart + off, len * sizeof(double), cudaMemcpyDefault, st));
    }
    for (kt_problem *p : gr->shards)
      if ((s = shard_finish(p, j, st)) != KT_OK) return s;
    return KT_OK;
  };
  if (update && (s = exchange(0)) != KT_OK) return s;
  for (int j = 1; j <= nt; ++j) {
    for (size_t i = 0; i < n; ++i)
      if ((s = fwd_step(gr->shards[i], update, st, false, a[i], j)) != KT_OK) return s;
    if (update && j < nt && (s = exchange(j)) != KT_OK) return s;
  }
  kt_status first = KT_OK;
  for (kt_problem *p : gr->shards) {
    s = read_status(p, st);
    if (s != KT_OK && first == KT_OK) first = s;
  }
  if (first != KT_OK) {
    for (kt_problem *p : gr->shards) p->have_fwd = p->have_bwd = false;
    return first;
  }
  for (kt_problem *p : gr->shards) commit_forward(p, update, false);
  return KT_OK;
}

// F over all shards' trajectories, summed in global trajectory order (as the unsharded problem does).
kt_status group_fidelity(kt_group *gr, double *F, cudaStream_t st) {
  double s = 0.0;
  int M = 0;
  for (kt_problem *p : gr->shards) {
    std::vector<KtCplx> tau(p->M);
    KT_CUDA(cudaMemcpyAsync(tau.data(), p->tau, sizeof(KtCplx) * p->M, cudaMemcpyDeviceToHost, st));
    KT_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < p->M; ++k) s += tau[k].re * tau[k].re + tau[k].im * tau[k].im;
    M += p->M;
  }
  *F = s / M;
  return KT_OK;
}

}  // namespace

extern "C" {

KT_API kt_status kt_nccl_unique_id(const char *nccl_library, void *id_out) {
  if (!id_out) return fail(KT_ERR_ARG, "NULL output");
  kt_status s = nccl_load(nccl_library);
  if (s != KT_OK) return s;
  const int r = g_nccl.get_unique_id(id_out);
  if (r != 0) return fail(KT_ERR_CUDA, "ncclGetUniqueId failed: %s", g_nccl.error_string(r));
  return KT_OK;
}

KT_API kt_status krotov_shard_nccl(kt_problem *p, const void *unique_id, int rank, int world, const char *nccl_library) {
  if (!p || !unique_id) return fail(KT_ERR_ARG, "NULL argument");
  if (!p->sharded) return fail(KT_ERR_ARG, "not a shard: create the problem with kt_config.M_total > 0");
  if (p->in_group) return fail(KT_ERR_STATE, "the shard belongs to a group");
  if (p->nccl_comm) return fail(KT_ERR_STATE, "the shard already has a communicator");
  if (world < 1 || rank < 0 || rank >= world || (long long)world * p->M != p->M_total ||
      p->tile_off * p->g.T != rank * p->M)
    return fail(KT_ERR_ARG, "NCCL shards hold equal slices in rank order: M_total = world * M, traj_offset = rank * M");
  kt_status s = nccl_load(nccl_library);
  if (s != KT_OK) return s;
  std::array<char, 128> id;
  std::memcpy(id.data(), unique_id, 128);
  void *comm = nullptr;
  const int r = g_nccl.comm_init_rank(&comm, world, id, rank);
  if (r != 0) return fail(KT_ERR_CUDA, "ncclCommInitRank failed: %s", g_nccl.error_string(r));
  p->nccl_comm = comm;
  p->nccl_rank = rank;
  p->nccl_world = world;
  return KT_OK;
}

KT_API kt_status krotov_group_init(kt_problem *const *shards, int n, kt_group **out) {
  if (!shards || !out || n < 1) return fail(KT_ERR_ARG, "NULL argument or n < 1");
  *out = nullptr;
  std::vector<kt_problem *> v(shards, shards + n);
  for (kt_problem *p : v)
    if (!p || !p->sharded || p->in_group || p->nccl_comm)
      return fail(KT_ERR_ARG, "every member must be a shard (M_total > 0) of no other group and without NCCL");
  std::sort(v.begin(), v.end(), [](const kt_problem *a, const kt_problem *b) { return a->tile_off < b->tile_off; });
  int next = 0;
  for (kt_problem *p : v) {
    const kt_problem *q = v[0];
    if (p->tile_off != next || p->M_total != q->M_total || p->n_tiles_total != q->n_tiles_total ||
        p->g.T != q->g.T || p->g.nthreads != q->g.nthreads || p->nt != q->nt || p->g.n_ctrl != q->g.n_ctrl)
      return fail(KT_ERR_ARG, "the shards must tile one problem: same M_total, tile width, nt and controls, "
                              "consecutive trajectory ranges");
    next += p->g.n_tiles;
  }
  if (next != v[0]->n_tiles_total) return fail(KT_ERR_ARG, "the shards do not cover all %d tiles", v[0]->n_tiles_total);
  kt_group *g = new kt_group();
  g->shards = v;
  for (kt_problem *p : v) p->in_group = true;
  *out = g;
  return KT_OK;
}

KT_API kt_status krotov_group_update(kt_group *gr, int n_iter, double *JT_out, void *stream) {
  if (!gr) return fail(KT_ERR_ARG, "NULL group");
  if (n_iter < 0) return fail(KT_ERR_ARG, "n_iter < 0");
  cudaStream_t st = (cudaStream_t)stream;
  kt_status s;
  bool fresh = false;
  for (kt_problem *p : gr->shards) fresh = fresh || !p->have_fwd;
  if (fresh && (s = group_forward(gr, 0, st)) != KT_OK) return s;
  for (int it = 0; it < n_iter; ++it) {
    for (kt_problem *p : gr->shards)
      if ((s = backward_sweep(p, st)) != KT_OK) return s;
    if ((s = group_forward(gr, 1, st)) != KT_OK) return s;
    if (JT_out) {
      double F = 0.0;
      if ((s = group_fidelity(gr, &F, st)) != KT_OK) return s;
      JT_out[it] = 1.0 - F;
    }
  }
  return KT_OK;
}

KT_API kt_status krotov_group_fidelity(kt_group *gr, double *F_out, void *stream) {
  if (!gr || !F_out) return fail(KT_ERR_ARG, "NULL argument");
  for (kt_problem *p : gr->shards)
    if (!p->have_fwd) return fail(KT_ERR_STATE, "no forward sweep yet");
  return group_fidelity(gr, F_out, (cudaStream_t)stream);
}

KT_API void krotov_group_free(kt_group *gr) {
  if (!gr) return;
  for (kt_problem *p : gr->shards) p->in_group = false;
  delete gr;
}

}  // extern "C"
