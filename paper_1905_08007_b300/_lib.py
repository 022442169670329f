"""ctypes binding of ``libqedmc.so`` (argument marshalling only).

Names follow the C ABI in include/qedmc.h.  Device buffers are torch CUDA
tensors (torch is used for device memory and streams only); every step of the
computation runs in the library's kernels.  If the library is missing the
import of the symbols raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from pathlib import Path

_HERE = Path(__file__).resolve().parent
MAX_LOOPS = 5

_ERRORS = {
    -1: "QED_EINVAL", -2: "QED_ENOMEM", -3: "QED_ECUDA", -4: "QED_ETIMEOUT",
    -5: "QED_EUNSTABLE_LIMIT", -6: "QED_ENOTFOUND",
}


class QedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Graph(C.Structure):
    _fields_ = [("n", C.c_int), ("pairs", C.c_int * (2 * MAX_LOOPS)), ("e", C.c_int),
                ("stream_id", C.c_uint32)]


class _Pdf(C.Structure):
    _fields_ = [("deg", C.POINTER(C.c_double)), ("c_div", C.c_double), ("d_min", C.c_double)]


class _BatchOpts(C.Structure):
    _fields_ = [("policy", C.c_int), ("rounds", C.c_int), ("chunk", C.c_uint64), ("use_graph", C.c_int),
                ("list_div", C.c_int), ("counter_base", C.c_uint64)]


class _Result(C.Structure):
    _fields_ = [("value", C.c_double), ("variance", C.c_double), ("sum_w", C.c_double * 2),
                ("sum_w2", C.c_double * 2), ("n", C.c_uint64), ("n_flagged", C.c_uint64),
                ("n_unstable", C.c_uint64), ("seconds", C.c_double),
                ("kernel_seconds", C.c_double), ("launches", C.c_uint32), ("dd_seconds", C.c_double),
                ("unstable_abs_w", C.c_double)]


@dataclass(frozen=True)
class Graph:
    """Vertex graph: photon a joins photon vertices pairs[a] = (s, t), the
    external vertex sits after e photon vertices; stream_id is the Philox
    counter word of its samples."""
    n: int
    pairs: tuple
    e: int
    stream_id: int = 0

    def _c(self):
        g = _Graph()
        g.n = self.n
        for a, (s, t) in enumerate(self.pairs):
            g.pairs[2 * a] = s
            g.pairs[2 * a + 1] = t
        g.e = self.e
        g.stream_id = self.stream_id
        return g

    @staticmethod
    def _from_c(g):
        return Graph(g.n, tuple((g.pairs[2 * a], g.pairs[2 * a + 1]) for a in range(g.n)), g.e, g.stream_id)


@dataclass
class Result:
    value: float
    variance: float
    sum_w: tuple
    sum_w2: tuple
    n: int
    n_flagged: int
    n_unstable: int
    seconds: float
    kernel_seconds: float = 0.0
    launches: int = 0
    dd_seconds: float = 0.0
    unstable_abs_w: float = 0.0

    @property
    def sigma(self):
        return self.variance ** 0.5

    def _c(self):
        r = _Result()
        r.value, r.variance = self.value, self.variance
        r.sum_w[0], r.sum_w[1] = self.sum_w
        r.sum_w2[0], r.sum_w2[1] = self.sum_w2
        r.n, r.n_flagged, r.n_unstable, r.seconds = self.n, self.n_flagged, self.n_unstable, self.seconds
        r.kernel_seconds, r.launches, r.dd_seconds = self.kernel_seconds, self.launches, self.dd_seconds
        r.unstable_abs_w = self.unstable_abs_w
        return r

    @staticmethod
    def _from_c(r):
        return Result(r.value, r.variance, (r.sum_w[0], r.sum_w[1]), (r.sum_w2[0], r.sum_w2[1]),
                      r.n, r.n_flagged, r.n_unstable, r.seconds, r.kernel_seconds, r.launches, r.dd_seconds,
                      r.unstable_abs_w)


_LIB = None


def lib_path() -> Path:
    return Path(os.environ.get("QEDMC_LIB", _HERE / "libqedmc.so"))


def load_library():
    """Load libqedmc.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = lib_path()
    if not p.exists():
        raise QedError(-3, f"{p} not built: run python -m paper_1905_08007_b300.build")
    L = C.CDLL(str(p))
    P = C.POINTER
    sig = {
        "qed_ctx_create": (C.c_int, [C.c_int, C.c_uint64, P(C.c_void_p)]),
        "qed_ctx_destroy": (C.c_int, [C.c_void_p]),
        "qed_ctx_set_stream": (C.c_int, [C.c_void_p, C.c_size_t]),
        "qed_ctx_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
        "qed_ctx_set_threshold": (C.c_int, [C.c_void_p, C.c_double]),
        "qed_last_error": (C.c_char_p, []),
        "qed_enumerate": (C.c_int, [C.c_int, C.c_int, P(_Graph), C.c_int, P(C.c_int)]),
        "qed_gauge_class": (C.c_int, [P(_Graph), C.c_int * 3]),
        "qed_diagram_load": (C.c_int, [C.c_void_p, P(_Graph), P(_Pdf), P(C.c_void_p)]),
        "qed_diagram_free": (C.c_int, [C.c_void_p]),
        "qed_diagram_info": (C.c_int, [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_double)]),
        "qed_integrate": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, P(_Result)]),
        "qed_integrate_range": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, P(_Result)]),
        "qed_dump_points": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
        "qed_eval_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, C.c_void_p]),
        "qed_result_merge": (C.c_int, [P(_Result), P(_Result), P(_Result)]),
        "qed_diagram_flops": (C.c_int, [C.c_void_p, P(C.c_double)]),
        "qed_diagram_flops_dd": (C.c_int, [C.c_void_p, P(C.c_double)]),
        "qed_pdf_grad": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, P(C.c_double),
                                   P(C.c_double)]),
        "qed_diagram_set_pdf_params": (C.c_int, [C.c_void_p, P(C.c_double), P(C.c_double)]),
        "qed_integrate_range_noalloc": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64,
                                                  P(_Result)]),
        "qed_integrate_batch": (C.c_int, [C.c_void_p, P(C.c_void_p), C.c_int, C.c_uint64, C.c_uint64,
                                          P(_BatchOpts), P(_Result)]),
        "qed_fp64_peak": (C.c_int, [C.c_int, C.c_double, P(C.c_double)]),
        "qed_diagram_calibrate_deg": (C.c_int, [C.c_void_p, C.c_int, C.c_uint64]),
        "qed_diagram_get_deg": (C.c_int, [C.c_void_p, P(C.c_double)]),
        "qed_programs_load": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t, P(C.c_int)]),
        "qed_ctx_set_vm": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
        "qed_ctx_set_rng": (C.c_int, [C.c_void_p, C.c_int]),
        "qed_ctx_set_flag_rule": (C.c_int, [C.c_void_p, C.c_int]),
        "qed_eval_interval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _check(rc):
    if rc != 0:
        raise QedError(rc, load_library().qed_last_error().decode())


def enumerate_graphs(n: int, reduced: bool = False):
    L = load_library()
    cnt = C.c_int(0)
    _check(L.qed_enumerate(n, int(reduced), None, 0, C.byref(cnt)))
    arr = (_Graph * cnt.value)()
    _check(L.qed_enumerate(n, int(reduced), arr, cnt.value, C.byref(cnt)))
    return [Graph._from_c(arr[i]) for i in range(cnt.value)]


def gauge_class(g: Graph):
    L = load_library()
    out = (C.c_int * 3)()
    cg = g._c()
    _check(L.qed_gauge_class(C.byref(cg), out))
    return tuple(out)


def fp64_peak(device: int = 0, ms: float = 50.0) -> float:
    """Measured FP64 FMA throughput of the device in FLOP/s."""
    v = C.c_double()
    _check(load_library().qed_fp64_peak(device, ms, C.byref(v)))
    return v.value


def merge_results(a: Result, b: Result) -> Result:
    L = load_library()
    ca, cb, co = a._c(), b._c(), _Result()
    _check(L.qed_result_merge(C.byref(ca), C.byref(cb), C.byref(co)))
    return Result._from_c(co)


QED_CTX_PREFER_PROGRAMS = 1
# generators of the sample points (qed_ctx_set_rng)
RNGS = {"philox": 0, "mrg32k3a": 1}
# which points the double-double pass re-evaluates (qed_ctx_set_flag_rule)
FLAG_RULES = {"estimate": 0, "interval": 1}


def program_files():
    """Bytecode integrand files written by the build (vm_n<n>.bin.z, zlib)."""
    return sorted((_HERE / "csrc" / "_gen").glob("vm_n*.bin.z"))


class Context:
    """qed_ctx: one CUDA device; owns the device buffers it allocates.

    The bytecode integrands the build wrote (four loops and up, and the
    lower orders for comparison) are registered on creation unless
    programs=False; prefer_programs=True makes graphs that also have a
    compiled integrand use their program (QED_CTX_PREFER_PROGRAMS)."""

    def __init__(self, device: int = 0, threads: int | None = None, blocks: int | None = None,
                 threshold: float | None = None, stream=None, programs: bool = True,
                 prefer_programs: bool = False, rng: str = "philox", flag_rule: str = "estimate"):
        L = load_library()
        self._h = C.c_void_p()
        _check(L.qed_ctx_create(device, QED_CTX_PREFER_PROGRAMS if prefer_programs else 0, C.byref(self._h)))
        self.device = device
        self.n_programs = 0
        self.vm_shape = (128, 1)
        if programs:
            import zlib
            for f in program_files():
                self.programs_load(zlib.decompress(f.read_bytes()))
        if threads is not None or blocks is not None:
            self.set_launch(threads or 256, blocks or 0)
        if threshold is not None:
            _check(L.qed_ctx_set_threshold(self._h, threshold))
        if stream is not None:
            self.set_stream(stream)
        self.rng = "philox"
        if rng != "philox":
            self.set_rng(rng)
        self.flag_rule = "estimate"
        if flag_rule != "estimate":
            self.set_flag_rule(flag_rule)

    def set_flag_rule(self, rule: str):
        """qed_ctx_set_flag_rule: "estimate" (FP64 rounding-error estimate) or
        "interval" (FP64 interval arithmetic, bytecode programs)."""
        if rule not in FLAG_RULES:
            raise QedError(-1, f"unknown flag rule {rule!r}")
        _check(load_library().qed_ctx_set_flag_rule(self._h, FLAG_RULES[rule]))
        self.flag_rule = rule

    def set_rng(self, rng: str):
        """qed_ctx_set_rng: "philox" (Philox4x32-10) or "mrg32k3a"."""
        if rng not in RNGS:
            raise QedError(-1, f"unknown generator {rng!r}")
        _check(load_library().qed_ctx_set_rng(self._h, RNGS[rng]))
        self.rng = rng

    def programs_load(self, data: bytes) -> int:
        """qed_programs_load: register the bytecode integrands of a program file."""
        cnt = C.c_int(0)
        _check(load_library().qed_programs_load(self._h, data, len(data), C.byref(cnt)))
        self.n_programs += cnt.value
        return cnt.value

    def set_vm(self, threads: int = 128, points: int = 1):
        """qed_ctx_set_vm: block size and points per thread of the interpreter kernels."""
        _check(load_library().qed_ctx_set_vm(self._h, threads, points))
        self.vm_shape = (threads, points)

    def set_launch(self, threads: int, blocks: int = 0):
        _check(load_library().qed_ctx_set_launch(self._h, threads, blocks))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream or a raw cudaStream_t integer."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(load_library().qed_ctx_set_stream(self._h, int(raw)))

    def load(self, g: Graph, deg=None, c_div: float = 0.0, d_min: float = 0.0) -> "Diagram":
        return Diagram(self, g, deg, c_div, d_min)

    def integrate_batch(self, diagrams, total_samples: int, seed: int = 0, policy: str = "variance",
                        rounds: int = 4, chunk: int = 1 << 18, use_graph: bool = True, list_div: int = 16,
                        counter_base: int = 0):
        """qed_integrate_batch: all graphs in one persistent launch per round,
        samples shared by running variance (policy "variance") or equally."""
        k = len(diagrams)
        arr = (C.c_void_p * k)(*[d._h.value for d in diagrams])
        o = _BatchOpts(0 if policy == "variance" else 1, rounds, chunk, 0 if use_graph else -1, list_div,
                       counter_base)
        out = (_Result * k)()
        _check(load_library().qed_integrate_batch(self._h, arr, k, int(total_samples), seed, C.byref(o), out))
        return [Result._from_c(out[i]) for i in range(k)]

    def close(self):
        if self._h:
            load_library().qed_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Diagram:
    """qed_diag: a loaded graph with its generated integrand and Eq. (1) tables."""

    def __init__(self, ctx: Context, g: Graph, deg=None, c_div=0.0, d_min=0.0):
        L = load_library()
        self.ctx = ctx
        self.graph = g
        self._h = C.c_void_p()
        pdf = _Pdf()
        self._deg_keep = None
        if deg is not None:
            import numpy as np
            arr = np.ascontiguousarray(np.asarray(deg, dtype=np.float64))
            self._deg_keep = arr
            pdf.deg = arr.ctypes.data_as(C.POINTER(C.c_double))
        pdf.c_div = c_div
        pdf.d_min = d_min
        cg = g._c()
        _check(L.qed_diagram_load(ctx._h, C.byref(cg), C.byref(pdf), C.byref(self._h)))
        nl, fid, lz = C.c_int(), C.c_int(), C.c_double()
        _check(L.qed_diagram_info(self._h, C.byref(nl), C.byref(fid), C.byref(lz)))
        self.n_lines, self.integrand_id, self.log_norm = nl.value, fid.value, lz.value

    def integrate(self, n_samples: int, seed: int = 0, begin: int = 0) -> Result:
        r = _Result()
        _check(load_library().qed_integrate_range(self._h, begin, n_samples, seed, C.byref(r)))
        return Result._from_c(r)

    def dump_points(self, begin: int, n: int, seed: int = 0):
        """(z [n, N], f [n], logp [n], flag [n]) as torch CUDA tensors."""
        import torch
        dev = torch.device("cuda", self.ctx.device)
        z = torch.empty((n, self.n_lines), dtype=torch.float64, device=dev)
        f = torch.empty(n, dtype=torch.float64, device=dev)
        lp = torch.empty(n, dtype=torch.float64, device=dev)
        fl = torch.empty(n, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize(dev)
        _check(load_library().qed_dump_points(self._h, begin, n, seed, z.data_ptr(), f.data_ptr(),
                                              lp.data_ptr(), fl.data_ptr()))
        return z, f, lp, fl

    def eval_points(self, z, prec: int = 0):
        """f at points z (torch CUDA float64 [n, N]) in FP64 (0) or DD (1)."""
        import torch
        z = z.contiguous()
        assert z.dtype == torch.float64 and z.is_cuda and z.shape[1] == self.n_lines
        f = torch.empty(z.shape[0], dtype=torch.float64, device=z.device)
        torch.cuda.synchronize(z.device)
        _check(load_library().qed_eval_points(self._h, z.data_ptr(), z.shape[0], prec, f.data_ptr()))
        return f

    def eval_interval(self, z):
        """qed_eval_interval: FP64 interval enclosure (lo, hi) at points z
        (torch CUDA float64 [n, N]); bytecode programs only."""
        import torch
        z = z.contiguous()
        assert z.dtype == torch.float64 and z.is_cuda and z.shape[1] == self.n_lines
        lo = torch.empty(z.shape[0], dtype=torch.float64, device=z.device)
        hi = torch.empty_like(lo)
        torch.cuda.synchronize(z.device)
        _check(load_library().qed_eval_interval(self._h, z.data_ptr(), z.shape[0], lo.data_ptr(), hi.data_ptr()))
        return lo, hi

    def calibrate_deg(self, n_base: int = 8, seed: int = 0):
        """Cap Deg(s) by the measured growth of the integrand in each limit."""
        _check(load_library().qed_diagram_calibrate_deg(self._h, n_base, seed))

    def deg_table(self):
        """The current Deg table as a list of 2^N floats."""
        out = (C.c_double * (1 << self.n_lines))()
        _check(load_library().qed_diagram_get_deg(self._h, out))
        return list(out)

    def flops_per_sample(self) -> float:
        v = C.c_double()
        _check(load_library().qed_diagram_flops(self._h, C.byref(v)))
        return v.value

    def flops_per_dd_sample(self) -> float:
        """qed_diagram_flops_dd: FP64 work of one double-double re-evaluation."""
        v = C.c_double()
        _check(load_library().qed_diagram_flops_dd(self._h, C.byref(v)))
        return v.value

    def close(self):
        if self._h:
            load_library().qed_diagram_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
