"""Python front end of liblret: a simulation handle, a circuit runner for the
shared op-list format, and a torch.autograd.Function around the adjoint.

Everything numeric runs in the CUDA library; this module converts arguments
(gate names to ABI calls, Pauli strings to bit masks, numpy arrays to pointers).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _ffi
from ._ffi import check, lib

_AXIS = {"x": 0, "y": 1, "z": 2}
_CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128)
_CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
# SWAP in the basis 2 b(q0) + b(q1)
_SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
_FIXED = {
    "x": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
    "s": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "t": np.array([[1, 0], [0, np.exp(0.25j * np.pi)]], dtype=np.complex128),
    "h": np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2.0),
}
_CHAN = {"dep": _ffi.LR_DEPOLARIZING, "ad": _ffi.LR_AMPLITUDE_DAMPING, "bf": _ffi.LR_BIT_FLIP}


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _cplx_flat(M):
    M = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
    return np.ascontiguousarray(M.view(np.float64).reshape(-1))


def pauli_masks(terms, n):
    """[(coeff, [(q, 'X'|'Y'|'Z'), ...]), ...] -> (xmask, zmask, coeff) arrays."""
    T = len(terms)
    xm = np.zeros(T, dtype=np.uint64)
    zm = np.zeros(T, dtype=np.uint64)
    cf = np.zeros(T, dtype=np.float64)
    for t, (c, string) in enumerate(terms):
        x = z = 0
        for q, s in string:
            if not 0 <= q < n:
                raise ValueError(f"qubit {q} out of range")
            if s in ("X", "Y"):
                x |= 1 << q
            if s in ("Z", "Y"):
                z |= 1 << q
        xm[t], zm[t], cf[t] = x, z, c
    return xm, zm, cf


def launch_count():
    """Kernels launched by the library so far in this process (lr_launch_count)."""
    return int(lib.lr_launch_count())


def kraus_preset(kind, p):
    out = np.zeros(32, dtype=np.float64)
    K = C.c_int(0)
    check(lib.lr_kraus_preset(_CHAN[kind], float(p), _dptr(out), C.byref(K)), "lr_kraus_preset")
    return out, K.value


class LRSim:
    """One low-rank simulation on the current CUDA device (rho = V V^dag)."""

    def __init__(self, n, r, dtype="c64", capacity=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("liblret needs a CUDA device")
        self.n, self.r = int(n), int(r)
        self.dtype = _ffi.LR_C64 if dtype in ("c64", "complex64", _ffi.LR_C64) else _ffi.LR_C128
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        cap = 4 * self.r if capacity is None else int(capacity)
        check(lib.lr_init_ex(self.n, self.r, self.dtype, cap, C.c_void_p(self.stream.cuda_stream),
                             C.byref(h)), "lr_init")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib.lr_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        check(lib.lr_reset(self.h), "lr_reset")

    def apply_gate(self, qubits, U, dU=None, param_id=-1):
        qs = (C.c_int * len(qubits))(*[int(q) for q in qubits])
        if isinstance(U, torch.Tensor) and U.is_cuda:
            # dense gate from a device matrix in the state's precision (lr_apply_gate_device)
            want = torch.complex64 if self.dtype == _ffi.LR_C64 else torch.complex128
            if U.dtype != want or not U.is_contiguous() or U.shape != (1 << len(qubits), 1 << len(qubits)):
                raise ValueError(f"device gate must be a contiguous {want} matrix of side 2^k")
            check(lib.lr_apply_gate_device(self.h, len(qubits), qs, C.c_void_p(U.data_ptr())),
                  "lr_apply_gate_device")
            return
        Uf = _cplx_flat(U)
        dUf = _cplx_flat(dU) if dU is not None else None
        check(lib.lr_apply_gate(self.h, len(qubits), qs, _dptr(Uf),
                                _dptr(dUf) if dUf is not None else None, int(param_id)), "lr_apply_gate")

    def apply_diagonal(self, qubits, d):
        """Diagonal gate: row x scaled by d[sum_i b(q_i) 2^(k-1-i)] (lr_apply_diagonal)."""
        qs = (C.c_int * len(qubits))(*[int(q) for q in qubits])
        df = _cplx_flat(np.asarray(d).reshape(-1))
        if df.size != 2 << len(qubits):
            raise ValueError("diagonal needs 2^k entries")
        check(lib.lr_apply_diagonal(self.h, len(qubits), qs, _dptr(df)), "lr_apply_diagonal")

    def apply_rotation(self, axis, q, theta, param_id=-1):
        check(lib.lr_apply_rotation(self.h, _AXIS[axis.lower()], int(q), float(theta), int(param_id)),
              "lr_apply_rotation")

    def apply_kraus(self, q, kraus):
        if isinstance(kraus, tuple) and len(kraus) == 2 and isinstance(kraus[0], np.ndarray) and kraus[0].dtype == np.float64:
            buf, K = kraus
        else:
            mats = [np.asarray(k, dtype=np.complex128) for k in kraus]
            K = len(mats)
            buf = np.zeros(32, dtype=np.float64)
            buf[: 8 * K] = _cplx_flat(np.stack(mats))
        check(lib.lr_apply_kraus(self.h, int(q), int(K), _dptr(buf)), "lr_apply_kraus")

    def apply_channel(self, kind, q, p):
        self.apply_kraus(q, kraus_preset(kind, p))

    def compress(self, r=0, want_discarded=False):
        if want_discarded:
            d = C.c_double(0.0)
            check(lib.lr_compress(self.h, int(r), C.byref(d)), "lr_compress")
            return d.value
        check(lib.lr_compress(self.h, int(r), None), "lr_compress")
        return None

    def set_eigensolver(self, which):
        """"auto", "jacobi", "tridiag" (one thread block) or "cluster" (8 thread blocks)."""
        check(lib.lr_set_eigensolver(self.h, {"auto": 0, "jacobi": 1, "tridiag": 2, "cluster": 3}[which]),
              "lr_set_eigensolver")

    def set_eig_precision(self, mode, iters=1):
        """Eigensolve of an FP32 state: "refined" (FP32 solve + FP64 refinement of the
        kept eigenvectors, `iters` correction steps; the default), "fp32" or "fp64"
        (lr_set_eig_precision)."""
        check(lib.lr_set_eig_precision(self.h, {"refined": 0, "fp32": 1, "fp64": 2}[mode], int(iters)),
              "lr_set_eig_precision")

    def last_eig(self):
        """(G, evals, evecs, k) of the last truncation's eigenproblem (lr_last_eig)."""
        m, k = C.c_int(0), C.c_int(0)
        G = np.zeros((256, 256), dtype=np.complex128)
        ev = np.zeros(256, dtype=np.float64)
        U = np.zeros((256, 256), dtype=np.complex128)
        check(lib.lr_last_eig(self.h, C.byref(m), C.byref(k), G.ctypes.data_as(C.POINTER(C.c_double)),
                              _dptr(ev), U.ctypes.data_as(C.POINTER(C.c_double))), "lr_last_eig")
        mm = m.value
        return (G.reshape(-1)[: mm * mm].reshape(mm, mm).copy(), ev[:mm].copy(),
                U.reshape(-1)[: mm * mm].reshape(mm, mm).copy(), k.value)

    def set_trunc_log(self, capacity=65536):
        """Record every truncation on the device (lr_set_trunc_log); 0 switches it off."""
        check(lib.lr_set_trunc_log(self.h, int(capacity)), "lr_set_trunc_log")
        self._tlog_cap = int(capacity)

    def trunc_log(self, group=1):
        """The truncations recorded since set_trunc_log / reset, one dict each: m, k,
        lambda_1, lambda_k, lambda_k1, discarded, trace, gap, and the intermediate rank
        of Eq. 8 for Kraus groups of `group` channels, V_I = (n / M)^(1/3) m (the column
        count m before a truncation is 4^M V for depolarizing groups)."""
        cnt = C.c_int64(0)
        check(lib.lr_get_trunc_log(self.h, None, 0, C.byref(cnt)), "lr_get_trunc_log")
        n = int(cnt.value)
        buf = np.zeros((max(n, 1), _ffi.LR_TRUNC_LOG_FIELDS), dtype=np.float64)
        check(lib.lr_get_trunc_log(self.h, _dptr(buf), n, C.byref(cnt)), "lr_get_trunc_log")
        keys = ("m", "k", "lambda_1", "lambda_k", "lambda_k1", "discarded", "trace", "gap")
        vi = (self.n / float(group)) ** (1.0 / 3.0)
        out = []
        stored = min(n, getattr(self, "_tlog_cap", 0))
        for row in buf[:stored]:
            d = dict(zip(keys, (float(x) for x in row)))
            d["m"], d["k"] = int(d["m"]), int(d["k"])
            d["V_I"] = vi * d["m"]
            out.append(d)
        return out

    def set_path(self, which):
        """"auto" (truncate without forming V' where possible) or "expand"."""
        check(lib.lr_set_path(self.h, {"auto": 0, "expand": 1}[which]), "lr_set_path")

    def set_tensor_cores(self, on=True):
        check(lib.lr_set_tensor_cores(self.h, 1 if on else 0), "lr_set_tensor_cores")

    def set_eps(self, eps):
        check(lib.lr_set_eps(self.h, float(eps)), "lr_set_eps")

    def probs(self, out=None):
        dt = torch.float32 if self.dtype == _ffi.LR_C64 else torch.float64
        if out is None:
            out = torch.empty(1 << self.n, dtype=dt, device="cuda")
        check(lib.lr_probs(self.h, C.c_void_p(out.data_ptr())), "lr_probs")
        return out

    def expect(self, terms):
        xm, zm, cf = pauli_masks(terms, self.n)
        return self.expect_masks(xm, zm, cf)

    def expect_masks(self, xm, zm, cf):
        out = C.c_double(0.0)
        check(lib.lr_expect(self.h, len(cf), xm.ctypes.data_as(C.POINTER(C.c_uint64)),
                            zm.ctypes.data_as(C.POINTER(C.c_uint64)), _dptr(cf), C.byref(out)), "lr_expect")
        return out.value

    def z_expect(self):
        out = np.zeros(self.n + 1, dtype=np.float64)
        check(lib.lr_z_expect(self.h, _dptr(out)), "lr_z_expect")
        return out[: self.n], out[self.n]

    def sample(self, uniforms):
        """Basis indices of len(uniforms) measurement shots drawn from Prob(x) by
        inverse transform with the caller's draws in [0, 1) (lr_sample)."""
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64).reshape(-1))
        out = np.zeros(len(u), dtype=np.int64)
        check(lib.lr_sample(self.h, len(u), _dptr(u), out.ctypes.data_as(C.POINTER(C.c_int64))), "lr_sample")
        return out

    def entropy(self):
        """(S in bits, effective rank 2^S) of the normalised state (lr_entropy)."""
        out = np.zeros(2, dtype=np.float64)
        check(lib.lr_entropy(self.h, _dptr(out)), "lr_entropy")
        return float(out[0]), float(out[1])

    def set_record(self, on=True):
        check(lib.lr_set_record(self.h, 1 if on else 0), "lr_set_record")

    def set_checkpoint(self, every):
        check(lib.lr_set_checkpoint(self.h, int(every)), "lr_set_checkpoint")

    def backward(self, terms, nparams):
        xm, zm, cf = pauli_masks(terms, self.n)
        g = np.zeros(max(nparams, 1), dtype=np.float64)
        check(lib.lr_backward(self.h, len(cf), xm.ctypes.data_as(C.POINTER(C.c_uint64)),
                              zm.ctypes.data_as(C.POINTER(C.c_uint64)), _dptr(cf), int(nparams), _dptr(g)),
              "lr_backward")
        return g[:nparams]

    def info(self):
        inf = _ffi.lr_info()
        st = lib.lr_get_info(self.h, C.byref(inf))
        if st not in (_ffi.LR_OK, _ffi.LR_ENOCONV):
            check(st, "lr_get_info")  # includes LR_ETIMEOUT from a tensor-core wait
        return {"n": inf.n, "columns": inf.columns, "capacity": inf.capacity, "dtype": inf.dtype,
                "compressions": inf.compressions, "stages": inf.stages, "discarded": inf.discarded,
                "last_gap": inf.last_gap, "converged": st == _ffi.LR_OK}

    def state(self):
        inf = self.info()
        dt = np.complex64 if self.dtype == _ffi.LR_C64 else np.complex128
        out = np.zeros((1 << self.n, inf["columns"]), dtype=dt)
        check(lib.lr_get_state(self.h, C.c_void_p(out.ctypes.data)), "lr_get_state")
        return out

    def set_timing(self, on=True):
        check(lib.lr_set_timing(self.h, 1 if on else 0), "lr_set_timing")

    def kernel_times(self):
        ms = np.zeros(_ffi.LR_NKCLASS, dtype=np.float64)
        cnt = np.zeros(_ffi.LR_NKCLASS, dtype=np.int64)
        check(lib.lr_kernel_times(self.h, _dptr(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))),
              "lr_kernel_times")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(_ffi.KCLASSES)}

    def last_eig_stats(self):
        sw = C.c_int(0)
        cyc = (C.c_longlong * 6)()
        check(lib.lr_last_eig_stats(self.h, C.byref(sw), cyc), "lr_last_eig_stats")
        return sw.value, list(cyc)

    def device_bytes(self):
        return int(lib.lr_device_bytes(self.h))


def is_gate(op):
    return op["op"] in ("rx", "ry", "rz", "cnot", "cz")


def run_ops(sim, ops, r=0, thetas=None, compress=True, group=1):
    """Apply an op list. A truncation follows every `group`-th channel (Kraus
    groups of M = group channels) and the circuit's last untruncated channels."""
    pending = 0
    for o in ops:
        name = o["op"]
        if name in ("rx", "ry", "rz"):
            pid = int(o.get("pid", -1))
            th = float(thetas[pid]) if (thetas is not None and pid >= 0) else float(o["theta"])
            sim.apply_rotation(name[1], o["q"], th, pid)
        elif name == "cnot":
            sim.apply_gate(o["q"], _CNOT)
        elif name == "cz":
            sim.apply_gate(o["q"], _CZ)
        elif name == "swap":
            sim.apply_gate(o["q"], _SWAP)
        elif name in _FIXED:
            sim.apply_gate([o["q"]], _FIXED[name])
        elif name == "unitary":
            sim.apply_gate(list(o["q"]), o["U"])
        elif name == "diag":
            sim.apply_diagonal(list(o["q"]), o["d"])
        elif name in _CHAN:
            sim.apply_channel(name, o["q"], o["p"] if "p" in o else o["gamma"])
            pending += 1
            if compress and pending == group:
                sim.compress(r)
                pending = 0
        else:
            raise ValueError(f"unknown op {name!r}")
    if compress and pending:
        sim.compress(r)
    return sim


class LRExpectation(torch.autograd.Function):
    """<H>(theta) of a parameterised noisy circuit; backward = liblret adjoint."""

    @staticmethod
    def forward(ctx, thetas, sim, ops, terms, r, ckpt_every):
        th = thetas.detach().cpu().numpy().astype(np.float64)
        sim.reset()
        sim.set_checkpoint(ckpt_every)
        sim.set_record(True)
        run_ops(sim, ops, r=r, thetas=th)
        val = sim.expect(terms)
        ctx.sim, ctx.terms, ctx.nparams = sim, terms, len(th)
        return torch.tensor(val, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.sim.backward(ctx.terms, ctx.nparams)
        ctx.sim.set_record(False)
        return torch.from_numpy(g) * grad_out, None, None, None, None, None


class LRBatch:
    """Many independent circuits advanced together (one CUDA graph per run).

    circuits: list of dicts {"n", "r", "ops"} in the shared op-list format.
    Semantics per circuit: truncation to rank r after every channel.
    """

    def __init__(self, circuits, dtype="c64", rows_per_split=0, use_graph=True, stream=None,
                 eig_precision="refined", eig_iters=1, splits=None, tensor_cores=True, cluster_min_m=None):
        """eig_precision (complex64): "refined" (FP32 solve + FP64 refinement of the kept
        eigenvectors), "fp32" or "fp64". splits: None or one Gram split count per
        circuit (0 = from rows_per_split), e.g. from autotune.BatchTable.splits_for.
        cluster_min_m: Gram matrices with at least this many rows go to the 8-CTA cluster
        eigensolver (0: none; None: the library's default)."""
        if not torch.cuda.is_available():
            raise RuntimeError("liblret needs a CUDA device")
        self.dtype = _ffi.LR_C64 if dtype in ("c64", "complex64", _ffi.LR_C64) else _ffi.LR_C128
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.circuits = circuits
        self._keep = []
        arr = (_ffi.lr_circuit * len(circuits))()
        for i, cd in enumerate(circuits):
            ops = (_ffi.lr_op * max(1, len(cd["ops"])))()
            for j, o in enumerate(cd["ops"]):
                qs = o["q"] if isinstance(o["q"], list) else [o["q"]]
                ops[j].kind = _ffi.OP_KIND[o["op"]]
                ops[j].q0 = int(qs[0])
                ops[j].q1 = int(qs[1]) if len(qs) > 1 else -1
                ops[j].theta = float(o.get("theta", 0.0))
                ops[j].p = float(o.get("p", o.get("gamma", 0.0)))
            self._keep.append(ops)
            arr[i].n, arr[i].r, arr[i].nops = int(cd["n"]), int(cd["r"]), len(cd["ops"])
            arr[i].ops = C.cast(ops, C.POINTER(_ffi.lr_op))
        opts = _ffi.lr_batch_opts()
        lib.lr_batch_opts_default(C.byref(opts))
        opts.dtype = self.dtype
        opts.eig_precision = {"refined": _ffi.LR_EIGP_REFINED, "fp32": _ffi.LR_EIGP_FP32,
                              "fp64": _ffi.LR_EIGP_FP64}[eig_precision]
        opts.eig_iters = int(eig_iters)
        opts.rows_per_split = int(rows_per_split)
        if splits is not None:
            if len(splits) != len(circuits):
                raise ValueError("splits needs one entry per circuit")
            sp = (C.c_int * len(circuits))(*[int(x) for x in splits])
            self._keep.append(sp)
            opts.splits = C.cast(sp, C.POINTER(C.c_int))
        opts.use_graph = 1 if use_graph else 0
        opts.tensor_cores = 1 if tensor_cores else 0
        if cluster_min_m is not None:
            opts.cluster_min_m = int(cluster_min_m)
        opts.stream = self.stream.cuda_stream
        h = C.c_void_p()
        check(lib.lr_batch_create_ex(arr, len(circuits), C.byref(opts), C.byref(h)), "lr_batch_create_ex")
        self.h = h

    def run(self):
        check(lib.lr_batch_run(self.h), "lr_batch_run")

    def reset(self):
        check(lib.lr_batch_reset(self.h), "lr_batch_reset")

    def info(self, i):
        inf = _ffi.lr_info()
        st = lib.lr_batch_info(self.h, int(i), C.byref(inf))
        if st not in (_ffi.LR_OK, _ffi.LR_ENOCONV):
            check(st, "lr_batch_info")
        return {"n": inf.n, "columns": inf.columns, "compressions": inf.compressions,
                "discarded": inf.discarded, "converged": st == _ffi.LR_OK}

    def probs(self, i):
        n = int(self.circuits[i]["n"])
        dt = torch.float32 if self.dtype == _ffi.LR_C64 else torch.float64
        out = torch.empty(1 << n, dtype=dt, device="cuda")
        check(lib.lr_batch_probs(self.h, int(i), C.c_void_p(out.data_ptr())), "lr_batch_probs")
        return out

    def stats(self):
        v = [C.c_int64() for _ in range(4)]
        check(lib.lr_batch_stats(self.h, *[C.byref(x) for x in v]), "lr_batch_stats")
        return dict(zip(["gates", "truncations", "steps", "launches"], [x.value for x in v]))

    def close(self):
        if getattr(self, "h", None):
            lib.lr_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
