"""Python binding of the C ABI: one ``Problem`` per optimisation problem.

Argument marshalling only; every step of the hot path runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _capi
from .model import NetworkFactors


def _c(arr, dtype=np.float64):
    a = np.ascontiguousarray(arr, dtype=dtype)
    return a


def _cplx(arr):
    """complex array -> contiguous float64 (re, im) pairs."""
    return np.ascontiguousarray(np.stack([np.real(arr), np.imag(arr)], axis=-1), dtype=np.float64)


def _ptr(a, ctype=ct.c_double):
    return a.ctypes.data_as(ct.POINTER(ctype)) if a is not None else None


def _check_dev(t, shape, name):
    """A contiguous float64 CUDA tensor of the given shape (device pointers cross the ABI as is)."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and tuple(t.shape) == tuple(shape)):
        raise ValueError(f"{name}: contiguous float64 CUDA tensor of shape {tuple(shape)} expected")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)   # torch.cuda.Stream


class Problem:
    """Trajectory-parallel Krotov optimisation of one network (C ABI ``kt_problem``).

    Parameters mirror ``kt_model_desc`` / ``kt_config``: ``eps_guess`` and ``shape`` are
    [n_ctrl, nt], ``lam`` [n_ctrl], ``uniforms`` [n_passes, M, draws_per_traj].
    ``precision`` is "fp64" or "fp32" (FP32-mixed: complex64 states, FP64 norms and sums).
    ``tile_traj``: 0 automatic, -1 autotuned at init, else trajectories per CTA tile.
    ``items_per_thread``: 0 automatic thread mapping, else the strided mapping with 1, 2, 4, 8 or 16
    items per thread.
    ``per_interval_launches``: False lets small problems run each sweep as one launch (info.whole_sweep);
    True keeps one launch per interval.
    ``update_rule``: "independent" (Eq. independent_traj_update) or "cross" (Eq. cross_traj_update).
    ``jump_scheme``: "bisection" (exact jump times) or "first_order" (at most one jump per interval).
    """

    def __init__(self, net: NetworkFactors, T: float, nt: int, M: int, eps_guess, shape, lam, uniforms,
                 precision: str = "fp64", ckpt_interval: int = 0, eps_bound: float = 0.0,
                 cheb_tol: float = 0.0, tile_traj: int = 0, psi0_batch=None, stream=None,
                 update_rule: str = "independent", jump_scheme: str = "bisection", ckpt_prefix: int = 0,
                 traj_offset: int = 0, M_total: int = 0, inject_copy_timeout: bool = False,
                 items_per_thread: int = 0, per_interval_launches: bool = False):
        self._lib = _capi.load()
        self.net = net
        self.T, self.nt, self.M = float(T), int(nt), int(M)
        self.n_ctrl = net.n_ctrl
        uniforms = _c(uniforms)
        if uniforms.ndim != 3 or uniforms.shape[1] != M:
            raise ValueError("uniforms must have shape [n_passes, M, draws_per_traj]")
        keep, md, cfg = _descriptors(net, self.T, self.nt, self.M, eps_guess, shape, lam, uniforms, precision,
                                     ckpt_interval, eps_bound, cheb_tol, tile_traj, psi0_batch, update_rule,
                                     jump_scheme, ckpt_prefix, traj_offset, M_total, inject_copy_timeout,
                                     items_per_thread, per_interval_launches)
        handle = ct.c_void_p()
        self._h = None
        _capi.check(self._lib.krotov_init(ct.byref(md), ct.byref(cfg), _stream_handle(stream), ct.byref(handle)),
                    "krotov_init")
        self._h = handle
        self._owned = True
        self.precision = precision
        self.info = self.get_info()

    @classmethod
    def _borrow(cls, handle, net, T, nt, M, precision):
        """View of a problem owned by a Batch (never freed through this object)."""
        self = cls.__new__(cls)
        self._lib = _capi.load()
        self.net = net
        self.T, self.nt, self.M = float(T), int(nt), int(M)
        self.n_ctrl = net.n_ctrl
        self._h = handle
        self._owned = False
        self.precision = precision
        self.info = self.get_info()
        return self

    # ------------------------------------------------------------------ calls
    def forward(self, update: bool = False, stream=None, keep_for_gradient: bool = False, want_F: bool = True):
        """One forward sweep; returns F (None with want_F=False: no host read of the fidelity).
        update: sequential Krotov update on the fly; keep_for_gradient: plain sweep that keeps the
        forward states for gradient()."""
        if update and keep_for_gradient:
            raise ValueError("a sweep either updates the pulse or keeps states for the gradient")
        mode = 1 if update else (2 if keep_for_gradient else 0)
        F = ct.c_double()
        _capi.check(self._lib.propagate_forward(self._h, mode, ct.byref(F) if want_F else None,
                                                _stream_handle(stream)), "propagate_forward")
        return F.value if want_F else None

    def gradient(self, eps=None, out=None, stream=None):
        """dJ_T/deps [n_ctrl, nt] as a CUDA float64 tensor (``out``, allocated if None), computed and
        written on the device.  eps None: at the current pulse with the jump record of the last
        forward(keep_for_gradient=True) held fixed; eps a CUDA float64 tensor [n_ctrl, nt]: the pulse
        is set from it and a forward sweep that keeps its states runs first."""
        import torch
        if out is None:
            out = torch.empty((self.n_ctrl, self.nt), dtype=torch.float64, device="cuda")
        _check_dev(out, (self.n_ctrl, self.nt), "out")
        e = None
        if eps is not None:
            _check_dev(eps, (self.n_ctrl, self.nt), "eps")
            e = ct.c_void_p(eps.data_ptr())
        _capi.check(self._lib.krotov_gradient(self._h, e, ct.c_void_p(out.data_ptr()), _stream_handle(stream)),
                    "krotov_gradient")
        return out

    def set_pulses_device(self, eps, stream=None) -> None:
        """Replace the pulse from a CUDA float64 tensor [n_ctrl, nt] (device-to-device, on stream)."""
        _check_dev(eps, (self.n_ctrl, self.nt), "eps")
        _capi.check(self._lib.krotov_set_pulses_device(self._h, ct.c_void_p(eps.data_ptr()), _stream_handle(stream)),
                    "krotov_set_pulses_device")

    def JT_device(self, out=None, stream=None):
        """J_T = 1 - F of the last forward sweep as a 0-d CUDA float64 tensor, written on the device."""
        import torch
        if out is None:
            out = torch.empty((), dtype=torch.float64, device="cuda")
        _check_dev(out, (), "out")
        _capi.check(self._lib.krotov_get_JT(self._h, ct.c_void_p(out.data_ptr()), _stream_handle(stream)),
                    "krotov_get_JT")
        return out

    def sweeps(self) -> int:
        """Forward sweeps completed since the problem was created (never reset)."""
        return int(self.get_info().sweeps)

    def backward(self, stream=None) -> None:
        _capi.check(self._lib.propagate_backward(self._h, _stream_handle(stream)), "propagate_backward")

    def update(self, n_iter: int = 1, stream=None):
        JT = np.zeros(n_iter)
        J = np.zeros(n_iter)
        _capi.check(self._lib.krotov_update(self._h, int(n_iter), _ptr(JT), _ptr(J), _stream_handle(stream)),
                    "krotov_update")
        return JT, J

    def fidelity(self):
        F = ct.c_double()
        tau = np.zeros((self.M, 2))
        _capi.check(self._lib.fidelity(self._h, ct.byref(F), _ptr(tau)), "fidelity")
        return F.value, tau[:, 0] + 1j * tau[:, 1]

    def pulses(self) -> np.ndarray:
        out = np.zeros((self.n_ctrl, self.nt))
        _capi.check(self._lib.krotov_get_pulses(self._h, _ptr(out)), "krotov_get_pulses")
        return out

    def deps(self) -> np.ndarray:
        out = np.zeros((self.n_ctrl, self.nt))
        _capi.check(self._lib.krotov_get_update(self._h, _ptr(out)), "krotov_get_update")
        return out

    def set_pulses(self, eps) -> None:
        e = _c(eps)
        _capi.check(self._lib.krotov_set_pulses(self._h, _ptr(e)), "krotov_set_pulses")

    def records(self):
        """list over trajectories of [(step, s, channel, c), ...] of the last forward sweep."""
        mj = self.info.max_jumps
        cnt = np.zeros(self.M, dtype=np.int32)
        st = np.zeros((self.M, mj), dtype=np.int32)
        ch = np.zeros((self.M, mj), dtype=np.int32)
        s = np.zeros((self.M, mj))
        c = np.zeros((self.M, mj))
        _capi.check(self._lib.krotov_get_records(self._h, _ptr(cnt, ct.c_int), _ptr(st, ct.c_int),
                                                 _ptr(ch, ct.c_int), _ptr(s), _ptr(c)), "krotov_get_records")
        return [[(int(st[k, m]), float(s[k, m]), int(ch[k, m]), float(c[k, m])) for m in range(cnt[k])]
                for k in range(self.M)]

    def states(self) -> np.ndarray:
        out = np.zeros((self.M, self.net.d, 2))
        _capi.check(self._lib.krotov_get_states(self._h, _ptr(out)), "krotov_get_states")
        return out[..., 0] + 1j * out[..., 1]

    def costate(self, j: int) -> np.ndarray:
        out = np.zeros((self.M, self.net.d, 2))
        _capi.check(self._lib.krotov_get_costate(self._h, int(j), _ptr(out)), "krotov_get_costate")
        return out[..., 0] + 1j * out[..., 1]

    def pulse_noise(self, ref=None, stream=None) -> np.ndarray:
        """nu_c = integral |e_c - smooth(e_c)| dt with e = current pulse (minus ``ref`` [n_ctrl, nt]
        when given), five-point cubic Savitzky-Golay smoothing; [n_ctrl]."""
        out = np.zeros(self.n_ctrl)
        r = _c(ref) if ref is not None else None
        _capi.check(self._lib.krotov_pulse_noise(self._h, _ptr(r), _ptr(out), _stream_handle(stream)),
                    "krotov_pulse_noise")
        return out

    def set_uniforms(self, uniforms, stream=None) -> None:
        """Replace the uniforms by a [n_passes, M, draws] block (pass counter restarts): a host array,
        or a CUDA float64 tensor (copied device to device)."""
        if hasattr(uniforms, "data_ptr") and getattr(uniforms, "is_cuda", False):
            if uniforms.dtype != __import__("torch").float64 or not uniforms.is_contiguous() or uniforms.dim() != 3:
                raise ValueError("uniforms: contiguous float64 CUDA tensor [n_passes, M, draws] expected")
            self._u_keep = uniforms
            ptr, n = ct.c_void_p(uniforms.data_ptr()), int(uniforms.shape[0])
        else:
            u = _c(uniforms)
            self._u_keep = u      # host buffer must outlive the asynchronous copy
            ptr, n = ct.c_void_p(u.ctypes.data), int(u.shape[0])
        _capi.check(self._lib.krotov_set_uniforms(self._h, ptr, n, _stream_handle(stream)), "krotov_set_uniforms")

    def set_profiling(self, on: bool = True) -> None:
        _capi.check(self._lib.krotov_set_profiling(self._h, int(bool(on))), "krotov_set_profiling")

    def profile(self):
        """{family: (total_ms, launches)} for the 'fwd' and 'bwd' interval kernels, the 'grad' kernel, the
        'cross' update kernels and the one-block update sums ('finish') since profiling was enabled."""
        ms = np.zeros(5)
        n = np.zeros(5, dtype=np.int64)
        _capi.check(self._lib.krotov_get_profile(self._h, _ptr(ms), n.ctypes.data_as(ct.POINTER(ct.c_longlong))),
                    "krotov_get_profile")
        return {"fwd": (float(ms[0]), int(n[0])), "bwd": (float(ms[1]), int(n[1])), "grad": (float(ms[2]), int(n[2])),
                "cross": (float(ms[3]), int(n[3])), "finish": (float(ms[4]), int(n[4]))}

    def shard_nccl(self, unique_id: bytes, rank: int, world: int, nccl_library: str = None) -> None:
        """Join the NCCL communicator of the problem's shards (this shard = ``rank`` of ``world``; the
        device must be current).  ``unique_id``: the 128 bytes of ``nccl_unique_id()`` from one rank."""
        uid = ct.create_string_buffer(bytes(unique_id), 128)
        _capi.check(self._lib.krotov_shard_nccl(self._h, uid, int(rank), int(world),
                                                nccl_library.encode() if nccl_library else None),
                    "krotov_shard_nccl")

    def checkpoint(self) -> dict:
        """What resumes this optimisation bit-identically: the current pulse, the pulse bound of the
        spectral estimate and the number of completed forward sweeps (pass p used uniforms row p).
        Resume with ``Problem(..., eps_guess=ck["eps"], eps_bound=ck["eps_bound"],
        uniforms=U[ck["passes"] - 1:])``, one ``forward()`` (it repeats the last sweep exactly, jump
        records included) and ``update()`` as before."""
        info = self.get_info()
        return {"eps": self.pulses(), "eps_bound": float(info.eps_bound), "passes": int(info.passes)}

    def get_info(self):
        info = _capi.Info()
        _capi.check(self._lib.krotov_get_info(self._h, ct.byref(info)), "krotov_get_info")
        return info

    def close(self) -> None:
        if self._h is not None:
            if self._owned:
                self._lib.krotov_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent problems whose Krotov iterations run as one CUDA graph launch each
    (C ABI ``kt_batch``).  ``specs`` is a list of dicts of ``Problem`` constructor arguments
    (net, T, nt, M, eps_guess, shape, lam, uniforms and the optional keywords)."""

    _KEYS = ("precision", "ckpt_interval", "eps_bound", "cheb_tol", "tile_traj", "psi0_batch", "update_rule",
             "jump_scheme", "ckpt_prefix", "items_per_thread", "per_interval_launches")

    def __init__(self, specs, stream=None):
        self._lib = _capi.load()
        self._h = None
        n = len(specs)
        keeps, mds, cfgs = [], [], []      # keeps: host arrays the descriptors point into
        for sp in specs:
            u = _c(sp["uniforms"])
            if u.ndim != 3 or u.shape[1] != int(sp["M"]):
                raise ValueError("uniforms must have shape [n_passes, M, draws_per_traj]")
            kw = {k: sp[k] for k in self._KEYS if k in sp}
            keep, md, cfg = _descriptors(sp["net"], float(sp["T"]), int(sp["nt"]), int(sp["M"]), sp["eps_guess"],
                                         sp["shape"], sp["lam"], u, **kw)
            keeps.append(keep)
            mds.append(md)
            cfgs.append(cfg)
        md_arr = (ct.POINTER(_capi.ModelDesc) * n)(*[ct.pointer(m) for m in mds])
        cfg_arr = (ct.POINTER(_capi.Config) * n)(*[ct.pointer(c) for c in cfgs])
        handle = ct.c_void_p()
        _capi.check(self._lib.krotov_init_batch(md_arr, cfg_arr, n, _stream_handle(stream), ct.byref(handle)),
                    "krotov_init_batch")
        self._h = handle
        self.problems = []
        for i, sp in enumerate(specs):
            ph = ct.c_void_p()
            _capi.check(self._lib.krotov_batch_problem(self._h, i, ct.byref(ph)), "krotov_batch_problem")
            self.problems.append(Problem._borrow(ph, sp["net"], sp["T"], sp["nt"], sp["M"],
                                                 sp.get("precision", "fp64")))

    def __len__(self):
        return len(self.problems)

    def update(self, n_iter: int = 1, stream=None) -> np.ndarray:
        """n_iter Krotov iterations of every problem; returns J_T = 1 - F as [n_iter, n_problems]."""
        JT = np.zeros((int(n_iter), len(self.problems)))
        _capi.check(self._lib.krotov_batch_update(self._h, int(n_iter), _ptr(JT), _stream_handle(stream)),
                    "krotov_batch_update")
        return JT

    def info(self) -> dict:
        n = ct.c_int()
        nodes = ct.c_longlong()
        nbytes = ct.c_longlong()
        _capi.check(self._lib.krotov_batch_info(self._h, ct.byref(n), ct.byref(nodes), ct.byref(nbytes)),
                    "krotov_batch_info")
        return {"n_problems": n.value, "graph_nodes": nodes.value, "device_bytes": nbytes.value}

    def close(self) -> None:
        if self._h is not None:
            for p in self.problems:
                p._h = None
            self._lib.krotov_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class DensityProblem(Problem):
    """Density-matrix Krotov optimisation of one network (Sec. 2.2, Eqs. krotovupdate,
    krotov_boundary; C ABI ``krotov_init_density``): rho runs forward under the master equation,
    P backward from |tgt><tgt| under its adjoint, and the pulse is updated sequentially by
    S/lambda Im <<P|[H_c, rho]>>.  The library propagates vec(rho) as one state of the 2N-node
    Liouville-space network, so the sweep calls are those of ``Problem``; ``rho()`` and ``P(j)``
    return d x d matrices.  The model's ``psi0`` is the (pure) initial state."""

    def __init__(self, net: NetworkFactors, T: float, nt: int, eps_guess, shape, lam, precision: str = "fp64",
                 ckpt_interval: int = 0, eps_bound: float = 0.0, cheb_tol: float = 0.0, stream=None,
                 ckpt_prefix: int = 0, per_interval_launches: bool = False):
        self._lib = _capi.load()
        self.net = net
        self.T, self.nt, self.M = float(T), int(nt), 1
        self.n_ctrl = net.n_ctrl
        dummy = np.full((1, 1, 1), -1.0)
        keep, md, cfg = _descriptors(net, self.T, self.nt, 1, eps_guess, shape, lam, dummy, precision,
                                     ckpt_interval, eps_bound, cheb_tol, 0, None, "independent", "bisection",
                                     ckpt_prefix, per_interval_launches=per_interval_launches)
        handle = ct.c_void_p()
        self._h = None
        _capi.check(self._lib.krotov_init_density(ct.byref(md), ct.byref(cfg), _stream_handle(stream),
                                                  ct.byref(handle)), "krotov_init_density")
        self._h = handle
        self._owned = True
        self.precision = precision
        self.info = self.get_info()

    def rho(self) -> np.ndarray:
        """rho(T) of the last forward sweep, d x d."""
        d = self.net.d
        out = np.zeros((1, d * d, 2))
        _capi.check(self._lib.krotov_get_states(self._h, _ptr(out)), "krotov_get_states")
        return (out[0, :, 0] + 1j * out[0, :, 1]).reshape(d, d)

    def P(self, j: int) -> np.ndarray:
        """Co-state P(t_j) of the last backward sweep, d x d (stored slots only)."""
        d = self.net.d
        out = np.zeros((1, d * d, 2))
        _capi.check(self._lib.krotov_get_costate(self._h, int(j), _ptr(out)), "krotov_get_costate")
        return (out[0, :, 0] + 1j * out[0, :, 1]).reshape(d, d)

    def records(self):
        return [[]]

    def states(self):
        raise AttributeError("a density-matrix problem has no trajectory states: use rho()")

    def costate(self, j):
        raise AttributeError("a density-matrix problem has no trajectory co-states: use P(j)")


def shard_ranges(M_total: int, world: int, tile: int = 1):
    """(traj_offset, M) of each of ``world`` shards of an M_total-trajectory problem: equal slices in
    rank order (what krotov_shard_nccl requires), each a whole number of tiles."""
    if world < 1 or M_total % world != 0 or (M_total // world) % tile != 0:
        raise ValueError(f"M_total = {M_total} does not split into {world} equal slices of whole {tile}-trajectory tiles")
    m = M_total // world
    return [(r * m, m) for r in range(world)]


def nccl_library_path():
    """The NCCL shared library that torch's CUDA build ships (NVIDIA's nccl wheel), or None to let the
    dynamic loader find libnccl.so.2."""
    import os
    try:
        import nvidia.nccl
        for d in list(getattr(nvidia.nccl, "__path__", [])):
            cand = os.path.join(d, "lib", "libnccl.so.2")
            if os.path.exists(cand):
                return cand
    except ImportError:
        pass
    return None


def nccl_unique_id(nccl_library: str = None) -> bytes:
    """A fresh NCCL unique id (128 bytes), created on one rank and sent to the others by the caller."""
    buf = ct.create_string_buffer(128)
    _capi.check(_capi.load().kt_nccl_unique_id(nccl_library.encode() if nccl_library else None, buf),
                "kt_nccl_unique_id")
    return buf.raw


class ShardGroup:
    """Shards of one problem (``Problem`` objects created with ``traj_offset``/``M_total``) driven
    together in this process on one stream (C ABI ``kt_group``): per interval the tile partials of the
    update overlap are copied between the shards before each forms Delta eps -- the exchange of a
    trajectory-sharded run, here without a network.  The shards stay owned by the caller."""

    def __init__(self, shards):
        self._lib = _capi.load()
        self.shards = list(shards)
        arr = (ct.c_void_p * len(self.shards))(*[p._h.value for p in self.shards])
        h = ct.c_void_p()
        self._h = None
        _capi.check(self._lib.krotov_group_init(arr, len(self.shards), ct.byref(h)), "krotov_group_init")
        self._h = h

    def update(self, n_iter: int = 1, stream=None) -> np.ndarray:
        JT = np.zeros(int(n_iter))
        _capi.check(self._lib.krotov_group_update(self._h, int(n_iter), _ptr(JT), _stream_handle(stream)),
                    "krotov_group_update")
        return JT

    def fidelity(self, stream=None) -> float:
        F = ct.c_double()
        _capi.check(self._lib.krotov_group_fidelity(self._h, ct.byref(F), _stream_handle(stream)),
                    "krotov_group_fidelity")
        return F.value

    def close(self) -> None:
        if self._h is not None:
            self._lib.krotov_group_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def bessel_j(alpha: float, n: int) -> np.ndarray:
    """J_0..J_{n-1}(alpha) from the library's Miller recurrence (host-side helper)."""
    out = np.zeros(n)
    _capi.check(_capi.load().kt_bessel_j(float(alpha), int(n), _ptr(out)), "kt_bessel_j")
    return out


_UPDATE_RULES = {"independent": 0, "cross": 1}
_JUMP_SCHEMES = {"bisection": 0, "first_order": 1}


def _descriptors(net, T, nt, M, eps_guess, shape, lam, uniforms, precision="fp64", ckpt_interval=0,
                 eps_bound=0.0, cheb_tol=0.0, tile_traj=0, psi0_batch=None, update_rule="independent",
                 jump_scheme="bisection", ckpt_prefix=0, traj_offset=0, M_total=0, inject_copy_timeout=False,
                 items_per_thread=0, per_interval_launches=False):
    """kt_model_desc / kt_config for ``net`` (the returned ``keep`` dict owns the host arrays)."""
    uniforms = _c(uniforms)
    keep = {
        "h0": _cplx(net.h0_local), "hc": _cplx(net.hc_local), "cn": _c(net.ctrl_node, np.int32),
        "a": _cplx(net.a_local), "pd": _c(net.pair_dst, np.int32), "ps": _c(net.pair_src, np.int32),
        "pc": _cplx(net.pair_coef), "lc": _cplx(net.lind_coef), "tgt": _cplx(net.psi_tgt),
        "psi0": _cplx(net.psi0) if psi0_batch is None else None,
        "psib": _cplx(psi0_batch) if psi0_batch is not None else None,
        "eps": _c(eps_guess), "shape": _c(shape), "lam": _c(lam), "U": uniforms,
    }
    md = _capi.ModelDesc(
        n_nodes=net.n_nodes, n_loc=net.n_loc, h0_local=_ptr(keep["h0"]),
        n_ctrl=net.n_ctrl, ctrl_node=_ptr(keep["cn"], ct.c_int), hc_local=_ptr(keep["hc"]),
        a_local=_ptr(keep["a"]), n_pairs=len(net.pair_dst),
        pair_dst=_ptr(keep["pd"], ct.c_int), pair_src=_ptr(keep["ps"], ct.c_int), pair_coef=_ptr(keep["pc"]),
        n_lind=net.lind_coef.shape[0], lind_coef=_ptr(keep["lc"]),
        psi0=_ptr(keep["psi0"]), psi0_batch=_ptr(keep["psib"]), psi_tgt=_ptr(keep["tgt"]))
    cfg = _capi.Config(
        T=float(T), nt=int(nt), M=int(M),
        prec=_capi.KT_FP64 if precision == "fp64" else _capi.KT_FP32_MIXED,
        ckpt_interval=int(ckpt_interval), eps_guess=_ptr(keep["eps"]), shape=_ptr(keep["shape"]),
        lambda_a=_ptr(keep["lam"]), uniforms=_ptr(keep["U"]), n_passes=uniforms.shape[0],
        draws_per_traj=uniforms.shape[2], eps_bound=float(eps_bound), cheb_tol=float(cheb_tol),
        tile_traj=int(tile_traj), update_rule=_UPDATE_RULES[update_rule], jump_scheme=_JUMP_SCHEMES[jump_scheme],
        ckpt_prefix=int(ckpt_prefix), traj_offset=int(traj_offset), M_total=int(M_total),
        inject_copy_timeout=int(bool(inject_copy_timeout)), items_per_thread=int(items_per_thread),
        per_interval_launches=int(bool(per_interval_launches)))
    return keep, md, cfg


def generator_dense(net, T, nt, M, eps_guess, shape, lam, uniforms, eps, direction=0, precision="fp64",
                    items_per_thread=0):
    """Dense generator expanded from the library's structured tables (host only): direction 0 gives
    H_eff(eps), direction 1 gives -H_eff(eps)^dag (d x d); directions 2 and 3 the same for the
    Liouville-space generator of a density-matrix problem (d^2 x d^2).  ``items_per_thread`` selects
    the thread mapping whose tables are expanded (the cavity-structure mapping re-slots its rows)."""
    keep, md, cfg = _descriptors(net, T, nt, M, eps_guess, shape, lam, uniforms, precision,
                                 items_per_thread=items_per_thread)
    d = net.d if direction < 2 else net.d ** 2
    out = np.zeros((d, d, 2))
    e = _c(eps)
    _capi.check(_capi.load().kt_generator_dense(ct.byref(md), ct.byref(cfg), int(direction), _ptr(e), _ptr(out)),
                "kt_generator_dense")
    return out[..., 0] + 1j * out[..., 1]
