"""B300 near-field direct sum of the Abacus N-body method (arXiv:1810.02916).

Thin ctypes binding over the C ABI in include/nearfield.h (libnearfield.so,
built in-tree by `paper_1810_02916_b300.build`).  This module only marshals
arguments: every step of the computation runs in the library's CUDA
kernels.  If the library is missing the import of any entry point fails with
an error; there is no CPU fallback.

Arrays may be NumPy arrays (host) or CUDA torch tensors (device); both are
passed to the library as plain pointers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnearfield.so")

NF_OK, NF_EINVAL, NF_ENOMEM, NF_ECUDA, NF_ETIMEOUT, NF_ESTATE = range(6)
PROFILE_WORDS = 34       # NF_PROFILE_WORDS of include/nearfield.h
ACC_COMPENSATED, ACC_PLAIN = 0, 1
SPLINE, PLUMMER = 0, 1
_STATUS = {1: "NF_EINVAL", 2: "NF_ENOMEM", 3: "NF_ECUDA", 4: "NF_ETIMEOUT", 5: "NF_ESTATE"}

EXPORTS = [
    "nf_create", "nf_destroy", "nf_last_error", "nf_set_stream", "nf_set_accumulation", "nf_bin_particles",
    "nf_set_particles", "nf_set_velocities", "nf_get_particles", "nf_num_particles", "nf_pair_count", "nf_forces",
    "nf_get_forces64", "nf_kick_drift", "nf_vjp", "nf_forces_batched", "nf_profile", "nf_profile_read",
    "nf_set_shape", "nf_tune", "nf_forces_noalloc", "nf_set_softening", "nf_spline_eps_from_plummer",
    "nf_choose_dt", "nf_multipoles", "nf_set_cutoff", "nf_generation", "nf_fail_allocations",
    "nf_profile_classes", "nf_set_tiling", "nf_get_tuning",
]


class NearFieldError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libnearfield.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_1810_02916_b300.build` "
                               "(the CUDA library is required; there is no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        p, i, i64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "nf_create": ([i, i, d, d, ctypes.POINTER(p)], i),
            "nf_destroy": ([p], None),
            "nf_last_error": ([p], ctypes.c_char_p),
            "nf_set_stream": ([p, p], i),
            "nf_set_accumulation": ([p, i], i),
            "nf_bin_particles": ([p, p, i64], i),
            "nf_set_particles": ([p, p, p, p, i64], i),
            "nf_set_velocities": ([p, p], i),
            "nf_get_particles": ([p, p, p, p, p, p], i),
            "nf_num_particles": ([p, ctypes.POINTER(i64)], i),
            "nf_pair_count": ([p, ctypes.POINTER(i64)], i),
            "nf_forces": ([p, p], i),
            "nf_get_forces64": ([p, p], i),
            "nf_kick_drift": ([p, d], i),
            "nf_vjp": ([p, p, p], i),
            "nf_forces_batched": ([ctypes.POINTER(p), i, ctypes.POINTER(p)], i),
            "nf_profile": ([p, i], i),
            "nf_profile_read": ([p, ctypes.POINTER(i64), ctypes.POINTER(d)], i),
            "nf_set_shape": ([p, i, i], i),
            "nf_tune": ([p, ctypes.c_char_p, i], i),
            "nf_forces_noalloc": ([i, d, d, p, p, i64, p, p, ctypes.c_char_p, i], i),
            "nf_set_softening": ([p, i], i),
            "nf_set_cutoff": ([p, ctypes.c_int64], i),
            "nf_choose_dt": ([p, d, d, ctypes.POINTER(d), ctypes.POINTER(d)], i),
            "nf_multipoles": ([p, i, p], i),
            "nf_spline_eps_from_plummer": ([d], d),
            "nf_generation": ([p, ctypes.POINTER(ctypes.c_uint64)], i),
            "nf_fail_allocations": ([i64, i64], i),
            "nf_profile_classes": ([p, p, i], i),
            "nf_set_tiling": ([p, i, i, i, i], i),
            "nf_get_tuning": ([p, p], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a) -> int | None:
    """Data pointer of a NumPy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check_arr(a, dtype, shape, name):
    if a is None:
        return
    dt = str(a.dtype).replace("torch.", "")
    if dt != np.dtype(dtype).name:
        raise TypeError(f"{name}: dtype {dt}, expected {np.dtype(dtype).name}")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {tuple(shape)}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class NearField:
    """One periodic box: cpd^3 cells, near-field radius R = 2, spline softening eps (box units)."""

    def __init__(self, cpd: int, eps: float, box: float = 1.0, R: int = 2):
        h = ctypes.c_void_p()
        rc = lib().nf_create(int(cpd), int(R), float(eps), float(box), ctypes.byref(h))
        if rc != NF_OK:
            raise NearFieldError(rc, lib().nf_last_error(None).decode())
        self._h = h
        self.cpd, self.eps, self.box, self.R = int(cpd), float(eps), float(box), int(R)

    # -------------------------------------------------------------- plumbing
    @property
    def handle(self):
        return self._h

    def _call(self, name, *args):
        rc = getattr(lib(), name)(self._h, *args)
        if rc != NF_OK:
            raise NearFieldError(rc, lib().nf_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().nf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        v = ctypes.c_int64()
        self._call("nf_num_particles", ctypes.byref(v))
        return int(v.value)

    @property
    def generation(self) -> int:
        """Changes whenever the box's particles change (load, kick-drift)."""
        v = ctypes.c_uint64()
        self._call("nf_generation", ctypes.byref(v))
        return int(v.value)

    @property
    def ncell(self) -> int:
        return self.cpd ** 3

    def set_stream(self, stream):
        self._call("nf_set_stream", _stream_handle(stream))

    def set_accumulation(self, mode: int):
        self._call("nf_set_accumulation", int(mode))

    def set_softening(self, mode: int):
        """SPLINE (compact spline, eps = eps_s) or PLUMMER (eps = eps_p)."""
        self._call("nf_set_softening", int(mode))

    def set_cutoff(self, n_min: int):
        """0: exact near field; >= 1024: far cells of >= n_min particles act through
        the quadrupoles of their 4^3 sub-cells (an approximation; see nf_set_cutoff)."""
        self._call("nf_set_cutoff", int(n_min))

    # -------------------------------------------------------------- particles
    def bin_particles(self, xyz):
        """Load global positions (n, 3) float64 in box units (NumPy or CUDA tensor)."""
        n = int(xyz.shape[0])
        _check_arr(xyz, np.float64, (n, 3), "xyz")
        self._call("nf_bin_particles", _ptr(xyz), n)

    def set_particles(self, cell_offsets, counts, pos):
        n = int(pos.shape[0])
        _check_arr(cell_offsets, np.int64, (self.ncell + 1,), "cell_offsets")
        _check_arr(counts, np.int32, (self.ncell,), "counts")
        _check_arr(pos, np.float32, (n, 4), "pos")
        self._call("nf_set_particles", _ptr(cell_offsets), _ptr(counts), _ptr(pos), n)

    def set_velocities(self, vel):
        _check_arr(vel, np.float32, (self.n, 4), "vel")
        self._call("nf_set_velocities", _ptr(vel))

    def get_particles(self):
        """State in storage order: offsets, counts, pos (n,4), vel (n,4), perm (n,) as NumPy arrays."""
        n = self.n
        out = dict(cell_offsets=np.empty(self.ncell + 1, np.int64), counts=np.empty(self.ncell, np.int32),
                   pos=np.empty((n, 4), np.float32), vel=np.empty((n, 4), np.float32), perm=np.empty(n, np.int64))
        self._call("nf_get_particles", _ptr(out["cell_offsets"]), _ptr(out["counts"]), _ptr(out["pos"]),
                   _ptr(out["vel"]), _ptr(out["perm"]))
        return out

    def pair_count(self) -> int:
        v = ctypes.c_int64()
        self._call("nf_pair_count", ctypes.byref(v))
        return int(v.value)

    # -------------------------------------------------------------- compute
    def forces(self, out=None):
        """Accelerations (n, 4) float32, box units, storage order.

        `out` may be a NumPy array or a CUDA tensor; None returns a new NumPy array.
        Pass out=False to keep the result in the box only (FP64 sums for kick-drift).
        """
        if out is False:
            self._call("nf_forces", None)
            return None
        if out is None:
            out = np.empty((self.n, 4), np.float32)
        _check_arr(out, np.float32, (self.n, 4), "out")
        self._call("nf_forces", _ptr(out))
        return out

    def forces64(self, out=None):
        if out is None:
            out = np.empty((self.n, 3), np.float64)
        _check_arr(out, np.float64, (self.n, 3), "out")
        self._call("nf_get_forces64", _ptr(out))
        if isinstance(out, np.ndarray):
            self.synchronize()
        return out

    def choose_dt(self, eta: float, dt_max: float):
        """(dt, {dt_acc, dt_drift, dt_max}) from the time-step criteria (Section 4.2.1)."""
        dt = ctypes.c_double()
        parts = (ctypes.c_double * 3)()
        self._call("nf_choose_dt", float(eta), float(dt_max), ctypes.byref(dt), parts)
        return float(dt.value), dict(dt_acc=parts[0], dt_drift=parts[1], dt_max=parts[2])

    def multipoles(self, order: int = 8, out=None):
        """Cartesian multipole moments of every cell, (cpd^3, (p+1)(p+2)(p+3)/6) float64, cell units."""
        T = (order + 1) * (order + 2) * (order + 3) // 6
        if out is None:
            out = np.empty((self.ncell, T), np.float64)
        _check_arr(out, np.float64, (self.ncell, T), "out")
        self._call("nf_multipoles", int(order), _ptr(out))
        return out

    def kick_drift(self, dt: float):
        self._call("nf_kick_drift", float(dt))

    def vjp(self, w, out=None):
        """d(sum_i w_i . a_i)/dx_k in box units, (n, 4) float32; w is (n, 4) float32."""
        _check_arr(w, np.float32, (self.n, 4), "w")
        if out is None:
            out = np.empty((self.n, 4), np.float32)
        _check_arr(out, np.float32, (self.n, 4), "out")
        self._call("nf_vjp", _ptr(w), _ptr(out))
        return out

    def synchronize(self):
        v = ctypes.c_int64()
        self._call("nf_num_particles", ctypes.byref(v))
        try:
            import torch
            if torch.cuda.is_available():
                torch.cuda.synchronize()
        except ImportError:
            pass

    # -------------------------------------------------------------- tuning / timing
    def profile(self, enable=True):
        """True / 1: event timing of the pair kernel; 2: also per-item-class clock sums (diagnostic)."""
        self._call("nf_profile", int(enable) if not isinstance(enable, bool) else (1 if enable else 0))

    PROFILE_KINDS = ("4-sink tiles", "2-sink tiles", "1-sink tiles", "split (<= 16 sinks)", "lane items")

    def profile_classes(self) -> dict:
        """Per-class sums of profile(2) since the last read: {class name: (cycles, items, pairs)} plus
        the warps' summed lifetimes and the kernel's wall span (ns)."""
        out = np.zeros(PROFILE_WORDS, np.uint64)
        self._call("nf_profile_classes", _ptr(out), PROFILE_WORDS)
        res = {}
        for cls in range(10):
            name = self.PROFILE_KINDS[cls // 2] + (" (piece)" if cls % 2 else "")
            res[name] = tuple(int(v) for v in out[3 * cls:3 * cls + 3])
        mx = np.iinfo(np.uint64).max
        start = int(mx - out[32]) if out[32] else 0
        res["warp_lifetime_cycles"] = int(out[30])
        res["warps"] = int(out[31])
        res["wall_ns"] = int(out[33]) - start if out[33] else 0
        return res

    def profile_read(self):
        """(launches, total ms) of the pair kernel since the last read."""
        k, ms = ctypes.c_int64(), ctypes.c_double()
        self._call("nf_profile_read", ctypes.byref(k), ctypes.byref(ms))
        return int(k.value), float(ms.value)

    def set_shape(self, warps: int, stage: int):
        self._call("nf_set_shape", int(warps), int(stage))

    def set_tiling(self, c4: int, c2: int, c1: int, split_floor: int):
        """Sink tiling of the work items and the split floor (see nf_set_tiling)."""
        self._call("nf_set_tiling", int(c4), int(c2), int(c1), int(split_floor))

    def tuning(self) -> dict:
        """Launch shape and sink tiling in use."""
        out = np.zeros(6, np.int32)
        self._call("nf_get_tuning", _ptr(out))
        return dict(warps=int(out[0]), stage=int(out[1]), c4=int(out[2]), c2=int(out[3]), c1=int(out[4]),
                    split_floor=int(out[5]))

    def tune(self) -> str:
        buf = ctypes.create_string_buffer(2048)
        self._call("nf_tune", buf, 2048)
        return buf.value.decode()


def fail_allocations(skip: int, count: int) -> None:
    """Test hook: after `skip` more device allocations, make the next `count` fail (NF_ENOMEM)."""
    rc = lib().nf_fail_allocations(int(skip), int(count))
    if rc != NF_OK:
        raise NearFieldError(rc, "nf_fail_allocations: skip and count must be >= 0")


def spline_eps_from_plummer(eps_plummer: float) -> float:
    """eps_s = 2.16 eps_p: equal minimum pairwise dynamical time (Section 4.3.1)."""
    return float(lib().nf_spline_eps_from_plummer(float(eps_plummer)))


def forces_batched(boxes, outs=None):
    """Forces of several boxes in one persistent launch; outs: list of arrays/tensors or None."""
    nb = len(boxes)
    harr = (ctypes.c_void_p * nb)(*[b.handle for b in boxes])
    if outs is None:
        outs = [np.empty((b.n, 4), np.float32) for b in boxes]
    oarr = (ctypes.c_void_p * nb)(*[_ptr(o) for o in outs])
    rc = lib().nf_forces_batched(harr, nb, oarr)
    if rc != NF_OK:
        raise NearFieldError(rc, lib().nf_last_error(boxes[0].handle).decode())
    return outs
