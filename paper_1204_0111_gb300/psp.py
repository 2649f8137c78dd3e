"""ctypes binding of libpsp (include/psp.h): argument marshalling only.

Every step of the method runs inside the library's CUDA kernels; this module
checks shapes and dtypes, passes raw pointers (torch CUDA tensors or host
numpy arrays) and the current CUDA stream, and turns status codes into
exceptions.  It fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libpsp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "psp.h")

PREC_C128, PREC_C64 = 0, 1
SI_MODES = {"extended": 0, "paper": 1, "none": 2, "two": 3}   # psp_si_mode
AUX_MOVING_PML, AUX_EXACT = 0, 1
STATUS = {0: "PSP_OK", 1: "PSP_ERR_ARG", 2: "PSP_ERR_OOM", 3: "PSP_ERR_CUDA", 4: "PSP_ERR_ZERO_PIVOT",
          5: "PSP_ERR_NOT_CONVERGED", 6: "PSP_ERR_TIMEOUT", 7: "PSP_ERR_STATE"}


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("pml_C", ctypes.c_double), ("alpha", ctypes.c_double), ("pad_depth", ctypes.c_int),
                ("leaf_size", ctypes.c_int), ("precision", ctypes.c_int), ("pml_faces", ctypes.c_int),
                ("aux_mode", ctypes.c_int), ("collect_stats", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("tc_min_dim", ctypes.c_int),
                ("sweep_level_tasks", ctypes.c_int), ("sweep_ctas_per_sm", ctypes.c_int),
                ("setup_temp_mb", ctypes.c_int), ("sweep_rhs_group", ctypes.c_int),
                ("solve_rhs_group", ctypes.c_int), ("sweep_min_rows", ctypes.c_int), ("test_sweep_stall", ctypes.c_int),
                ("gmres_basis", ctypes.c_int),
                ("factor_every_panel", ctypes.c_int), ("panel_begin", ctypes.c_int), ("panel_count", ctypes.c_int),
                ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p), ("alloc_ctx", ctypes.c_void_p),
                ("selective_inversion", ctypes.c_int), ("c64_diag_fp64", ctypes.c_int),
                ("sweep_max_rows", ctypes.c_int), ("sweep_claim_ahead", ctypes.c_int)]


# psp_options.dev_alloc / dev_free callback types
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("extra_flops", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("applies", ctypes.c_int), ("relres_max", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("status_front", ctypes.c_int), ("groups", ctypes.c_int), ("min_pivot_abs", ctypes.c_double),
                ("reserved", ctypes.c_int * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class SweepTuning(ctypes.Structure):
    _fields_ = [("sweep_level_tasks", ctypes.c_int), ("sweep_ctas_per_sm", ctypes.c_int),
                ("sweep_rhs_group", ctypes.c_int), ("candidates", ctypes.c_int), ("initial_ms", ctypes.c_double),
                ("best_ms", ctypes.c_double), ("sweep_min_rows", ctypes.c_int), ("sweep_max_rows", ctypes.c_int),
                ("sweep_claim_ahead", ctypes.c_int), ("reserved", ctypes.c_int * 1)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class SetupTuning(ctypes.Structure):
    _fields_ = [("selective_inversion", ctypes.c_int), ("tc_min_dim", ctypes.c_int), ("candidates", ctypes.c_int),
                ("setup_ms", ctypes.c_double), ("apply_ms", ctypes.c_double), ("initial_total_ms", ctypes.c_double),
                ("best_total_ms", ctypes.c_double), ("reserved", ctypes.c_int * 4)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["selective_inversion"] = {v: k for k, v in SI_MODES.items()}[d["selective_inversion"]]
        return d


class PSPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int


def header_functions():
    """Names of every function declared in include/psp.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(psp_[a-z_]+)\s*\(", text)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libpsp.so is not built ({LIB_PATH}); run `python -m paper_1204_0111_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "psp_default_options": (None, [ctypes.POINTER(Options)]),
        "psp_setup": (_I, [ctypes.POINTER(Grid), _P, ctypes.c_double, _I, _I, ctypes.POINTER(Options), _P,
                           ctypes.POINTER(_P)]),
        "psp_setup_batch": (_I, [_I, ctypes.POINTER(Grid), ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(Options), _P,
                                 ctypes.POINTER(_P)]),
        "psp_batch_layout": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64), _I]),
        "psp_apply": (_I, [_P, _P, _P, _I, _P]),
        "psp_apply_noalloc": (_I, [_P, _P, _P, _I, _P]),
        "psp_matvec": (_I, [_P, _I, _P, _P, _I, _P]),
        "psp_solve": (_I, [_P, _P, _P, _I, ctypes.c_double, _I, _I, ctypes.POINTER(SolveInfo), _P]),
        "psp_symbolic_export": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t)]),
        "psp_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "psp_export_front": (_I, [_P, _I, _I, _P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
        "psp_export_second_inverse": (_I, [_P, _I, _I, _P, ctypes.POINTER(_I)]),
        "psp_stats": (_I, [_P, ctypes.POINTER(KernelStat), _I, ctypes.POINTER(_I), _I]),
        "psp_tune_sweep": (_I, [_P, _I, _I, _P, ctypes.POINTER(SweepTuning)]),
        "psp_check_status": (_I, [_P, _P]),
        "psp_tune_setup": (_I, [_P, _I, _I, _P, ctypes.POINTER(SetupTuning)]),
        "psp_sweep_part": (_I, [_P, _P, _I, _I, _P]),
        "psp_solve_history": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
        "psp_plan_panels": (_I, [ctypes.POINTER(Grid), _I, _I, ctypes.POINTER(Options), ctypes.POINTER(_I),
                                 ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double), _I, ctypes.POINTER(_I)]),
        "psp_destroy": (_I, [_P]),
        "psp_status_string": (ctypes.c_char_p, [_I]),
        "psp_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != 0:
        raise PSPError(status, lib().psp_last_error().decode())


def _ptr_and_len(a, complex_=True):
    """(pointer, element count) of a contiguous torch tensor or numpy array."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = torch.complex128 if complex_ else torch.float64
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"expected a contiguous {want} tensor, got {a.dtype}")
            return a.data_ptr(), a.numel()
    except ImportError:
        pass
    want = np.complex128 if complex_ else np.float64
    if not isinstance(a, np.ndarray) or a.dtype != want or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous {np.dtype(want)} array")
    return a.ctypes.data, a.size


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


class SweepingPreconditioner:
    """Handle over psp_setup / psp_apply / psp_solve (Algs. 1.4, 1.5 and GMRES(k) of §2.4)."""

    def __init__(self, c, h, omega, gamma, panel_depth, pad=None, leaf=64, pml_C=4.0, alpha=2 * math.pi,
                 precision="c128", faces=63, mode="moving", stream=None, collect_stats=0, tensor_cores=True,
                 tc_min_dim=0, sweep_level_tasks=0, sweep_ctas_per_sm=0, setup_temp_mb=0, sweep_rhs_group=0,
                 solve_rhs_group=0, test_sweep_stall=0, gmres_basis="auto", factor_every_panel=False,
                 panels=None, allocator=None, selective_inversion="extended", sweep_min_rows=0,
                 diag_fp64=False, sweep_max_rows=0, sweep_claim_ahead=0):
        nz, ny, nx = c.shape
        self.nx, self.ny, self.nz = nx, ny, nz
        self.N = nx * ny * nz
        self.points = [self.N]
        g = Grid(nx, ny, nz, float(h))
        o = _options(pad, leaf, pml_C, alpha, precision, faces, mode, collect_stats, tensor_cores, tc_min_dim,
                     sweep_level_tasks, sweep_ctas_per_sm, setup_temp_mb, sweep_rhs_group, solve_rhs_group)
        o.test_sweep_stall = int(test_sweep_stall)
        o.sweep_min_rows = int(sweep_min_rows)
        o.c64_diag_fp64 = 1 if diag_fp64 else 0
        o.sweep_max_rows = int(sweep_max_rows)
        o.sweep_claim_ahead = int(sweep_claim_ahead)
        o.gmres_basis = {"auto": 0, "z": 1, "v": 2}[gmres_basis]
        o.factor_every_panel = 1 if factor_every_panel else 0
        if panels is not None:                   # (first, count): one block of a multi-GPU sweep
            o.panel_begin, o.panel_count = int(panels[0]), int(panels[1])
        o.selective_inversion = SI_MODES[selective_inversion]
        if allocator is not None:                # (alloc(bytes) -> int, free(int)): the caller owns device memory
            self._alloc_cbs = _allocator_callbacks(*allocator)
            o.dev_alloc = ctypes.cast(self._alloc_cbs[0], ctypes.c_void_p)
            o.dev_free = ctypes.cast(self._alloc_cbs[1], ctypes.c_void_p)
        cp, n = _ptr_and_len(c, complex_=False)
        if n != self.N:
            raise ValueError("c has the wrong size")
        self._keep = c
        h_ = _P()
        st = lib().psp_setup(ctypes.byref(g), cp, float(omega), int(gamma), int(panel_depth), ctypes.byref(o),
                             _stream(stream), ctypes.byref(h_))
        self._finish(h_, st)

    def _finish(self, h_, st):
        self._h = h_
        if st != 0:
            msg = lib().psp_last_error().decode()
            self.close()
            raise PSPError(st, msg)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().psp_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _nrhs(self, a):
        _, n = _ptr_and_len(a)
        if n % self.N:
            raise ValueError("vector block size is not a multiple of N")
        return n // self.N

    def apply(self, rhs, out, stream=None):
        nr = self._nrhs(rhs)
        if self._nrhs(out) != nr:
            raise ValueError("rhs and out differ in size")
        _check(lib().psp_apply(self._h, _ptr_and_len(rhs)[0], _ptr_and_len(out)[0], nr, _stream(stream)))
        return out

    def matvec(self, x, y, which=0, stream=None):
        nr = self._nrhs(x)
        _check(lib().psp_matvec(self._h, int(which), _ptr_and_len(x)[0], _ptr_and_len(y)[0], nr, _stream(stream)))
        return y

    def solve(self, f, u, tol=1e-5, k=20, maxit=500, stream=None, raise_on_nonconvergence=True):
        nr = self._nrhs(f)
        info = SolveInfo()
        st = lib().psp_solve(self._h, _ptr_and_len(f)[0], _ptr_and_len(u)[0], nr, float(tol), int(k), int(maxit),
                             ctypes.byref(info), _stream(stream))
        if st != 0 and (raise_on_nonconvergence or st != 5):
            _check(st)
        return info.as_dict()

    def solve_history(self, kind=0):
        """psp_solve_history: (rows, cols) array of the last solve's residuals; kind 0 per iteration (Arnoldi
        estimate), kind 1 per restart cycle (true residual)."""
        r, c = _I(), _I()
        _check(lib().psp_solve_history(self._h, int(kind), None, 0, ctypes.byref(r), ctypes.byref(c)))
        buf = (ctypes.c_double * max(r.value * c.value, 1))()
        _check(lib().psp_solve_history(self._h, int(kind), buf, r.value * c.value, ctypes.byref(r), ctypes.byref(c)))
        return np.frombuffer(buf, dtype=np.float64)[:r.value * c.value].reshape(r.value, c.value).copy()

    def sweep_part(self, u, direction, stream=None):
        """psp_sweep_part: the forward (0) or backward (1) half of Alg. 1.5 over this handle's block, in place."""
        nr = self._nrhs(u)
        _check(lib().psp_sweep_part(self._h, _ptr_and_len(u)[0], nr, int(direction), _stream(stream)))
        return u

    def tune_setup(self, nrhs=1, expected_applies=20, stream=None):
        """psp_tune_setup: re-factor under each candidate setup and keep the cheapest for the expected solve."""
        t = SetupTuning()
        _check(lib().psp_tune_setup(self._h, int(nrhs), int(expected_applies), _stream(stream), ctypes.byref(t)))
        return t.as_dict()

    def check_status(self, stream=None):
        """psp_check_status: raise PSPError(PSP_ERR_TIMEOUT) if a sweep wait gave up since the last check."""
        _check(lib().psp_check_status(self._h, _stream(stream)))

    def info(self):
        m = _I()
        nf = ctypes.c_int64()
        fb = ctypes.c_int64()
        _check(lib().psp_info(self._h, ctypes.byref(m), ctypes.byref(nf), ctypes.byref(fb)))
        return {"panels": m.value, "fronts": nf.value, "factor_bytes": fb.value}

    def stats(self, reset=False):
        """{kernel: {launches, total_ms, flops, bytes}} accumulated by this handle (psp_stats)."""
        n = _I()
        _check(lib().psp_stats(self._h, None, 0, ctypes.byref(n), 0))
        buf = (KernelStat * max(n.value, 1))()
        _check(lib().psp_stats(self._h, buf, n.value, ctypes.byref(n), 1 if reset else 0))
        return {buf[i].name.decode(): {"launches": buf[i].launches, "total_ms": buf[i].total_ms,
                                       "flops": buf[i].flops, "bytes": buf[i].bytes,
                                       "extra_flops": buf[i].extra_flops} for i in range(n.value)}

    def tune_sweep(self, nrhs=1, reps=3, stream=None):
        """psp_tune_sweep: time candidate sweep schedules on this handle, keep the fastest."""
        t = SweepTuning()
        _check(lib().psp_tune_sweep(self._h, int(nrhs), int(reps), _stream(stream), ctypes.byref(t)))
        return t.as_dict()

    def symbolic(self, panel):
        n = ctypes.c_size_t()
        _check(lib().psp_symbolic_export(self._h, int(panel), None, ctypes.byref(n)))
        buf = (ctypes.c_int32 * n.value)()
        _check(lib().psp_symbolic_export(self._h, int(panel), buf, ctypes.byref(n)))
        return np.frombuffer(buf, dtype=np.int32).copy()

    def export_front(self, panel, sn):
        s = _I()
        u = _I()
        _check(lib().psp_export_front(self._h, int(panel), int(sn), None, ctypes.byref(s), ctypes.byref(u)))
        out = np.zeros(((s.value + u.value) * s.value,), dtype=np.complex128)
        _check(lib().psp_export_front(self._h, int(panel), int(sn), out.ctypes.data, ctypes.byref(s), ctypes.byref(u)))
        return out.reshape(s.value, s.value + u.value).T, s.value, u.value

    def export_second_inverse(self, panel, sn):
        """The two-inverse form's second inverse of L_TL of one front (s x s, built row by row)."""
        s = _I()
        _check(lib().psp_export_second_inverse(self._h, int(panel), int(sn), None, ctypes.byref(s)))
        out = np.zeros((s.value * s.value,), dtype=np.complex128)
        _check(lib().psp_export_second_inverse(self._h, int(panel), int(sn), out.ctypes.data, ctypes.byref(s)))
        return out.reshape(s.value, s.value).T


class SweepingPreconditionerBatch(SweepingPreconditioner):
    """Handle over psp_setup_batch: independent problems factored, swept and solved together.

    ``problems`` is a list of dicts with keys c (nz, ny, nx), h, omega, gamma, panel_depth; the other
    keyword arguments are the shared options of SweepingPreconditioner.  Vectors are batched blocks
    (see pack / unpack): problem q's N_q x nrhs block after problem q-1's."""

    def __init__(self, problems, pad=None, leaf=64, pml_C=4.0, alpha=2 * math.pi, precision="c128", faces=63,
                 mode="moving", stream=None, collect_stats=0, tensor_cores=True, tc_min_dim=0, sweep_level_tasks=0,
                 sweep_ctas_per_sm=0, setup_temp_mb=0, sweep_rhs_group=0, solve_rhs_group=0,
                 selective_inversion="extended", factor_every_panel=False, allocator=None, sweep_max_rows=0,
                 sweep_claim_ahead=0):
        n = len(problems)
        grids = (Grid * n)()
        cs = (_P * n)()
        om = (ctypes.c_double * n)()
        ga = (_I * n)()
        de = (_I * n)()
        self._keep = []
        self.points = []
        for q, pr in enumerate(problems):
            c = pr["c"]
            nz, ny, nx = c.shape
            grids[q] = Grid(nx, ny, nz, float(pr["h"]))
            cp, cnt = _ptr_and_len(c, complex_=False)
            if cnt != nx * ny * nz:
                raise ValueError("c has the wrong size")
            cs[q] = cp
            om[q] = float(pr["omega"])
            ga[q] = int(pr["gamma"])
            de[q] = int(pr["panel_depth"])
            self._keep.append(c)
            self.points.append(nx * ny * nz)
        self.N = sum(self.points)
        o = _options(pad, leaf, pml_C, alpha, precision, faces, mode, collect_stats, tensor_cores, tc_min_dim,
                     sweep_level_tasks, sweep_ctas_per_sm, setup_temp_mb, sweep_rhs_group, solve_rhs_group)
        o.selective_inversion = SI_MODES[selective_inversion]
        o.factor_every_panel = 1 if factor_every_panel else 0
        o.sweep_max_rows = int(sweep_max_rows)
        o.sweep_claim_ahead = int(sweep_claim_ahead)
        if allocator is not None:
            self._alloc_cbs = _allocator_callbacks(*allocator)
            o.dev_alloc = ctypes.cast(self._alloc_cbs[0], ctypes.c_void_p)
            o.dev_free = ctypes.cast(self._alloc_cbs[1], ctypes.c_void_p)
        h_ = _P()
        st = lib().psp_setup_batch(n, grids, cs, om, ga, de, ctypes.byref(o), _stream(stream), ctypes.byref(h_))
        self._finish(h_, st)
        if st == 0:
            m = _I()
            pts = (ctypes.c_int64 * n)()
            _check(lib().psp_batch_layout(self._h, ctypes.byref(m), pts, n))
            assert m.value == n and list(pts) == self.points

    def offsets(self, nrhs):
        """Start of each problem's block in a batched vector block with nrhs right-hand sides."""
        out, o = [], 0
        for n in self.points:
            out.append(o)
            o += n * nrhs
        return out

    def pack(self, blocks):
        """[(nrhs, N_q) arrays or tensors] -> one flat batched block."""
        try:
            import torch
            if isinstance(blocks[0], torch.Tensor):
                return torch.cat([b.reshape(-1) for b in blocks])
        except ImportError:
            pass
        return np.concatenate([np.asarray(b).reshape(-1) for b in blocks])

    def unpack(self, flat, nrhs):
        """Flat batched block -> [(nrhs, N_q) views]."""
        return [flat[o:o + n * nrhs].reshape(nrhs, n) for o, n in zip(self.offsets(nrhs), self.points)]


def _allocator_callbacks(alloc, free):
    """ctypes callbacks for psp_options.dev_alloc / dev_free around Python callables (kept alive by
    the handle).  alloc(bytes) returns a device address (int) or 0; free(address) releases it."""
    def a(nbytes, _ctx):
        try:
            return int(alloc(int(nbytes)) or 0)
        except Exception:
            return 0

    def f(ptr, _ctx):
        free(int(ptr))

    return ALLOC_FN(a), FREE_FN(f)


def _options(pad, leaf, pml_C, alpha, precision, faces, mode, collect_stats, tensor_cores, tc_min_dim,
             sweep_level_tasks, sweep_ctas_per_sm, setup_temp_mb, sweep_rhs_group=0, solve_rhs_group=0):
    o = Options()
    lib().psp_default_options(ctypes.byref(o))
    o.pml_C = float(pml_C)
    o.alpha = float(alpha)
    o.pad_depth = -1 if pad is None else int(pad)
    o.leaf_size = int(leaf)
    o.precision = {"c128": PREC_C128, "c64": PREC_C64}[precision]
    o.pml_faces = int(faces)
    o.aux_mode = {"moving": AUX_MOVING_PML, "exact": AUX_EXACT}[mode]
    o.collect_stats = int(collect_stats)
    o.tensor_cores = 1 if tensor_cores else 0
    o.tc_min_dim = int(tc_min_dim)
    o.sweep_level_tasks = int(sweep_level_tasks)
    o.sweep_ctas_per_sm = int(sweep_ctas_per_sm)
    o.setup_temp_mb = int(setup_temp_mb)
    o.sweep_rhs_group = int(sweep_rhs_group)
    o.solve_rhs_group = int(solve_rhs_group)
    return o


def parse_symbolic(buf):
    """Decode psp_symbolic_export's int32 stream into (meta, [(s, u, parent, nodes, struct), ...])."""
    nx, ny, nz, lead, nsn = (int(v) for v in buf[:5])
    p = 5
    sns = []
    for _ in range(nsn):
        s, u, par = (int(v) for v in buf[p:p + 3])
        p += 3
        nodes = buf[p:p + s].copy()
        p += s
        struct = buf[p:p + u].copy()
        p += u
        sns.append((s, u, par, nodes, struct))
    return {"nx": nx, "ny": ny, "nz": nz, "lead": lead, "nsn": nsn}, sns


def plan_panels(nx, ny, nz, h, gamma, panel_depth, pad=None, leaf=64, mode="moving"):
    """psp_plan_panels (host only): [(z0, z1), ...] of the m panels and each panel's setup flops."""
    o = _options(pad, leaf, 4.0, 2 * math.pi, "c128", 63, mode, 0, True, 0, 0, 0, 0)
    g = Grid(int(nx), int(ny), int(nz), float(h))
    m = _I()
    _check(lib().psp_plan_panels(ctypes.byref(g), int(gamma), int(panel_depth), ctypes.byref(o), None, None, None, 0,
                                 ctypes.byref(m)))
    z0 = (_I * m.value)()
    z1 = (_I * m.value)()
    cost = (ctypes.c_double * m.value)()
    _check(lib().psp_plan_panels(ctypes.byref(g), int(gamma), int(panel_depth), ctypes.byref(o), z0, z1, cost, m.value,
                                 ctypes.byref(m)))
    return [(z0[i], z1[i]) for i in range(m.value)], [cost[i] for i in range(m.value)]
