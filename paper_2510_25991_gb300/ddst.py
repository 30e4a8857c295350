"""Python binding of the C ABI (same names; argument marshalling only).

Arrays may be CUDA ``torch`` tensors (device pointers) or contiguous NumPy / CPU tensors
(host pointers, staged by the library).  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib as L

__all__ = ["DDSTError", "ddst_options_default", "ddst_setup", "ddst_setup_batch",
           "ddst_build_transfer", "ddst_compress", "ddst_compress_hbs", "HBS", "ddst_solve", "ddst_solve_batch", "ddst_march",
           "ddst_solve_adjoint", "ddst_solve_adjoint_batch", "ddst_interface_trace",
           "ddst_get_transfer", "ddst_apply_interface", "ddst_query", "ddst_get_precision",
           "ddst_time_apply", "ddst_get_options", "ddst_solve_interface",
           "ddst_autotune", "ddst_autotune_key", "ddst_autotune_lookup", "ddst_autotune_store",
           "ddst_partition",
           "ddst_residual_noalloc",
           "ddst_kernel_launches",
           "ddst_last_error",
           "ddst_destroy", "Solver", "DDSTSolve"]


class DDSTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.name = L.STATUS_NAMES.get(status, str(status))


def _ptr(x):
    """Address of a contiguous FP64 array (torch tensor on any device, or NumPy array)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("arrays must be contiguous float64")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float64")
        return x.ctypes.data
    raise TypeError(type(x))


def _check_sizes(prob, **arrays):
    """Element counts of interior (f, u, dL/du, dL/df) and nodal (g, a, dL/dg, dL/da) arrays of
    one problem: the library takes plain pointers and cannot check them itself."""
    d, n = prob["dim"], prob["n"]
    nodal = {"g", "a", "c", "dLdg", "dLda"}
    for name, x in arrays.items():
        if x is None:
            continue
        k = x.numel() if hasattr(x, "data_ptr") else np.asarray(x).size
        want = (n + 1) ** d if name in nodal else (n - 1) ** d
        if k != want:
            raise ValueError(f"{name} has {k} entries; a {d}D problem with n = {n} needs {want}")


def _check(lib, ctx, st):
    if st != L.DDST_OK:
        msg = lib.ddst_last_error(ctx)
        raise DDSTError(st, msg.decode() if msg else "")


_PRECISIONS = {"fp64": L.DDST_FP64, "mixed": L.DDST_MIXED, "mixed_tf32": L.DDST_MIXED_TF32,
               "auto": L.DDST_AUTO}


def ddst_options_default(**overrides):
    """The library's default options with ``overrides`` applied; ``precision`` may be given as
    "fp64", "mixed", "mixed_tf32" or "auto".  Unknown option names raise TypeError (a ctypes structure would
    otherwise take them silently as plain attributes)."""
    lib = L.load()
    o = L.ddst_options()
    lib.ddst_options_default(C.byref(o))
    fields = {f[0] for f in L.ddst_options._fields_}
    for k, v in overrides.items():
        if k not in fields:
            raise TypeError(f"unknown option {k!r}; options are {', '.join(sorted(fields))}")
        if k == "precision" and isinstance(v, str):
            if v.lower() not in _PRECISIONS:
                raise ValueError(f"precision must be one of {', '.join(_PRECISIONS)}, not {v!r}")
            v = _PRECISIONS[v.lower()]
        if k == "autotune_cache" and v is not None:
            v = os.fsencode(v)  # the structure keeps the bytes object alive
        setattr(o, k, v)
    return o


def _options_dict(o):
    d = {k: getattr(o, k) for k, _ in L.ddst_options._fields_}
    d["precision"] = {L.DDST_FP64: "fp64", L.DDST_MIXED: "mixed", L.DDST_MIXED_TF32: "mixed_tf32",
                      L.DDST_AUTO: "auto"}.get(d["precision"], d["precision"])
    if d["autotune_cache"] is not None:
        d["autotune_cache"] = os.fsdecode(d["autotune_cache"])
    return d


def _coeffs(a, b=(0.0, 0.0, 0.0), c=None):
    cf = L.ddst_coeffs()
    cf.a = _ptr(a)
    bb = list(b) + [0.0] * (3 - len(b))
    cf.b = (C.c_double * 3)(*bb[:3])
    cf.c = _ptr(c)
    return cf


def ddst_setup(dim, n, a, slab_width, b=(0.0, 0.0, 0.0), c=None, options=None, stream=None):
    """Returns an opaque context handle (c_void_p)."""
    lib = L.load()
    g = L.ddst_grid(dim, n)
    cf = _coeffs(a, b, c)
    out = C.c_void_p()
    st = lib.ddst_setup(C.byref(g), C.byref(cf), int(slab_width),
                        C.byref(options) if options is not None else None,
                        C.c_void_p(stream) if stream else None, C.byref(out))
    _check(lib, None, st)
    return out


def ddst_setup_batch(problems, options=None, stream=None):
    """``problems``: list of dicts with ``dim, n, w, a`` and optional ``b, c``."""
    lib = L.load()
    k, grids, coeffs, widths = _problem_arrays(problems)
    out = C.c_void_p()
    st = lib.ddst_setup_batch(k, grids, coeffs, widths,
                              C.byref(options) if options is not None else None,
                              C.c_void_p(stream) if stream else None, C.byref(out))
    _check(lib, None, st)
    return out


def ddst_build_transfer(ctx):
    lib = L.load()
    _check(lib, ctx, lib.ddst_build_transfer(ctx))


def ddst_compress(ctx, tol):
    lib = L.load()
    _check(lib, ctx, lib.ddst_compress(ctx, float(tol)))


def ddst_compress_hbs(ctx, rank, oversample=10):
    """Nested-basis HBS form of every transfer operator, rank ``rank`` from ``3 rank +
    oversample`` Gaussian samples (Sec. 2.4, Alg. 1)."""
    lib = L.load()
    _check(lib, ctx, lib.ddst_compress_hbs(ctx, int(rank), int(oversample)))


class HBS:
    """A dense operator compressed on its own into HBS form (``ddst_hbs_create``).

    ``S``: ng x ng float64 NumPy array; ``omega``, ``psi``: ng x nsamples float64 NumPy arrays
    or None (drawn on the device); ``precision``: "fp64" or "mixed"."""

    def __init__(self, S, rank, nsamples=None, leaf=None, omega=None, psi=None, precision="fp64"):
        lib = L.load()
        S = np.ascontiguousarray(S, dtype=np.float64)
        ng = S.shape[0]
        if S.shape != (ng, ng):
            raise ValueError("S must be square")
        nsamples = 3 * rank + 10 if nsamples is None else int(nsamples)
        leaf = 2 * rank if leaf is None else int(leaf)
        keep = [S]
        po = pp = None
        if omega is not None or psi is not None:
            omega = np.ascontiguousarray(omega, dtype=np.float64)
            psi = np.ascontiguousarray(psi, dtype=np.float64)
            if omega.shape != (ng, nsamples) or psi.shape != (ng, nsamples):
                raise ValueError("omega and psi must be ng x nsamples")
            keep += [omega, psi]
            po, pp = omega.ctypes.data, psi.ctypes.data
        self.ng = ng
        self.h = C.c_void_p()
        st = lib.ddst_hbs_create(S.ctypes.data, ng, int(rank), nsamples, leaf, po, pp,
                                 _PRECISIONS[precision], C.byref(self.h))
        _check(lib, None, st)

    def apply(self, x, y, transpose=False):
        lib = L.load()
        _check(lib, None, lib.ddst_hbs_apply(self.h, _ptr(x), _ptr(y), int(bool(transpose))))

    def dense(self):
        lib = L.load()
        out = np.empty((self.ng, self.ng))
        _check(lib, None, lib.ddst_hbs_expand(self.h, out.ctypes.data))
        return out

    def stats(self):
        """(tree depth L, stored numbers)."""
        lib = L.load()
        lv, ne = C.c_int(), C.c_int64()
        _check(lib, None, lib.ddst_hbs_stats(self.h, C.byref(lv), C.byref(ne)))
        return lv.value, ne.value

    def close(self):
        if self.h:
            L.load().ddst_hbs_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ddst_solve(ctx, f, g, u, raise_on_error=True):
    lib = L.load()
    info = L.ddst_info()
    st = lib.ddst_solve(ctx, _ptr(f), _ptr(g), _ptr(u), C.byref(info))
    if raise_on_error:
        _check(lib, ctx, st)
    return st, info.as_dict()


def _parr(xs):
    return (C.c_void_p * len(xs))(*[_ptr(x) for x in xs])


def ddst_solve_batch(ctx, fs, gs, us, raise_on_error=True):
    lib = L.load()
    info = L.ddst_info()
    st = lib.ddst_solve_batch(ctx, _parr(fs), _parr(gs), _parr(us), C.byref(info))
    if raise_on_error:
        _check(lib, ctx, st)
    return st, info.as_dict()


def ddst_march(ctx, nsteps, dt, vels, u0s, us, raise_on_error=True):
    """IMEX backward-Euler marching: ``vels[q]`` (dim, (n+1)^dim) nodal velocity, ``u0s[q]`` the
    interior initial state, ``us[q]`` receives the state after ``nsteps`` steps."""
    lib = L.load()
    info = L.ddst_info()
    st = lib.ddst_march(ctx, int(nsteps), float(dt), _parr(vels), _parr(u0s), _parr(us),
                        C.byref(info))
    if raise_on_error:
        _check(lib, ctx, st)
    return st, info.as_dict()


def ddst_solve_adjoint(ctx, dLdu, dLdf=None, dLdg=None, dLda=None, raise_on_error=True):
    lib = L.load()
    info = L.ddst_info()
    st = lib.ddst_solve_adjoint(ctx, _ptr(dLdu), _ptr(dLdf), _ptr(dLdg), _ptr(dLda), C.byref(info))
    if raise_on_error:
        _check(lib, ctx, st)
    return st, info.as_dict()


def ddst_solve_adjoint_batch(ctx, dLdus, dLdfs, dLdgs, dLdas, raise_on_error=True):
    lib = L.load()
    info = L.ddst_info()
    st = lib.ddst_solve_adjoint_batch(ctx, _parr(dLdus), _parr(dLdfs), _parr(dLdgs),
                                      _parr(dLdas), C.byref(info))
    if raise_on_error:
        _check(lib, ctx, st)
    return st, info.as_dict()


def ddst_interface_trace(ctx, prob, out):
    lib = L.load()
    _check(lib, ctx, lib.ddst_interface_trace(ctx, prob, _ptr(out)))


def ddst_get_transfer(ctx, prob, j, side, out):
    lib = L.load()
    _check(lib, ctx, lib.ddst_get_transfer(ctx, prob, j, side, _ptr(out)))


def ddst_apply_interface(ctx, prob, x, y, transpose=False):
    lib = L.load()
    _check(lib, ctx, lib.ddst_apply_interface(ctx, prob, _ptr(x), _ptr(y), int(bool(transpose))))


def ddst_solve_interface(ctx, prob, rhs, x, transpose=False):
    """x = (I - K)^{-1} rhs (or ^{-T}) for one problem by the direct (block cyclic reduction)
    interface solver."""
    lib = L.load()
    _check(lib, ctx, lib.ddst_solve_interface(ctx, prob, _ptr(rhs), _ptr(x), int(bool(transpose))))


def ddst_time_apply(ctx, transpose=False, reps=50):
    """Mean device milliseconds of one interface-operator application (diagnostic)."""
    lib = L.load()
    ms = C.c_float()
    _check(lib, ctx, lib.ddst_time_apply(ctx, int(bool(transpose)), int(reps), C.byref(ms)))
    return ms.value


def ddst_query(ctx, prob=0):
    lib = L.load()
    nds, ng, mr = C.c_int(), C.c_int64(), C.c_int()
    # the context is const here: its errors are reported in the process-wide message
    _check(lib, None, lib.ddst_query(ctx, prob, C.byref(nds), C.byref(ng), C.byref(mr)))
    return nds.value, ng.value, mr.value


def ddst_get_precision(ctx):
    """"fp64", "mixed" or "mixed_tf32": the arithmetic the context was set up with (what "auto"
    chose)."""
    lib = L.load()
    p = C.c_int()
    _check(lib, None, lib.ddst_get_precision(ctx, C.byref(p)))
    return {L.DDST_FP64: "fp64", L.DDST_MIXED_TF32: "mixed_tf32"}.get(p.value, "mixed")


def ddst_residual_noalloc(dim, n, a, f, g, u, r, norms, b=(0.0, 0.0, 0.0), c=None, stream=None):
    """Allocation-free FP64 residual r = b(f, g) - A u and norms (||r||, ||b||); device arrays
    only.  The library receives plain pointers and cannot see array sizes, so they are checked
    here before anything is launched (ValueError).  ``stream`` defaults to torch's current CUDA
    stream when the arrays are torch tensors (else the legacy default stream).  The call returns
    once the work is enqueued: synchronize that stream before reading r or norms."""
    _check_sizes(dict(dim=dim, n=n), f=f, g=g, u=u, r=r, a=a, c=c)
    k = norms.numel() if hasattr(norms, "data_ptr") else np.asarray(norms).size
    if k < 2:
        raise ValueError(f"norms has {k} entries; it needs 2")
    if stream is None and hasattr(u, "data_ptr") and getattr(u, "is_cuda", False):
        import torch
        stream = torch.cuda.current_stream(u.device).cuda_stream
    lib = L.load()
    grid = L.ddst_grid(dim, n)
    cf = _coeffs(a, b, c)
    st = lib.ddst_residual_noalloc(C.byref(grid), C.byref(cf), _ptr(f), _ptr(g), _ptr(u), _ptr(r),
                                   _ptr(norms), C.c_void_p(stream) if stream else None)
    _check(lib, None, st)


def ddst_get_options(ctx):
    """The options the context runs with (automatic choices resolved, tuned knobs applied)."""
    lib = L.load()
    o = L.ddst_options()
    _check(lib, None, lib.ddst_get_options(ctx, C.byref(o)))
    return _options_dict(o)


def _problem_arrays(problems):
    k = len(problems)
    grids = (L.ddst_grid * k)(*[L.ddst_grid(p["dim"], p["n"]) for p in problems])
    coeffs = (L.ddst_coeffs * k)(*[_coeffs(p["a"], p.get("b") or (0.0,) * 3, p.get("c"))
                                   for p in problems])
    widths = (C.c_int * k)(*[int(p["w"]) for p in problems])
    return k, grids, coeffs, widths


def ddst_autotune(problems, fs, gs, compress_tol=0.0, solves_per_setup=1, stream=None, **opts):
    """Times the schedule knobs left automatic in ``opts`` on these problems and right-hand
    sides; returns the report as a dict (``chosen`` is an options dict).  With
    ``autotune_cache=path`` the choice is stored there for later setups."""
    if isinstance(problems, dict):
        problems, fs, gs = [problems], [fs], [gs]
    for p, f, g in zip(problems, fs, gs):
        _check_sizes(p, f=f, g=g, a=p["a"], c=p.get("c"))
    lib = L.load()
    k, grids, coeffs, widths = _problem_arrays(problems)
    o = ddst_options_default(**opts)
    rep = L.ddst_tune_report()
    st = lib.ddst_autotune(k, grids, coeffs, widths, _parr(fs), _parr(gs), float(compress_tol),
                           int(solves_per_setup), C.byref(o), C.c_void_p(stream) if stream else None,
                           C.byref(rep))
    _check(lib, None, st)
    d = {k2: getattr(rep, k2) for k2, _ in L.ddst_tune_report._fields_ if k2 != "chosen"}
    d["chosen"] = _options_dict(rep.chosen)
    return d


def ddst_autotune_key(problems, precision="mixed"):
    if isinstance(problems, dict):
        problems = [problems]
    lib = L.load()
    k, grids, coeffs, widths = _problem_arrays(problems)
    buf = C.create_string_buffer(8192)
    prec = _PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib, None, lib.ddst_autotune_key(k, grids, coeffs, widths, prec, buf, len(buf)))
    return buf.value.decode()


def ddst_autotune_lookup(path, key, **opts):
    """(found, options dict): the cached knobs applied to ``opts``' automatic fields."""
    lib = L.load()
    o = ddst_options_default(**opts)
    found = C.c_int()
    _check(lib, None, lib.ddst_autotune_lookup(os.fsencode(path), key.encode(), C.byref(o),
                                               C.byref(found)))
    return bool(found.value), _options_dict(o)


def ddst_autotune_store(path, key, **opts):
    lib = L.load()
    o = ddst_options_default(**opts)
    _check(lib, None, lib.ddst_autotune_store(os.fsencode(path), key.encode(), C.byref(o)))


def ddst_partition(costs, world):
    """(owner per item, load per rank): the library's deterministic sharding of independent
    items over ``world`` ranks."""
    lib = L.load()
    k = len(costs)
    cost = (C.c_double * max(k, 1))(*[float(c) for c in costs])
    owner = (C.c_int * max(k, 1))()
    load = (C.c_double * world)()
    _check(lib, None, lib.ddst_partition(k, cost, int(world), owner, load))
    return [owner[i] for i in range(k)], [load[r] for r in range(world)]


def ddst_kernel_launches():
    return int(L.load().ddst_kernel_launches())


def ddst_last_error(ctx=None):
    lib = L.load()
    m = lib.ddst_last_error(ctx)
    return m.decode() if m else ""


def ddst_destroy(ctx):
    if ctx:
        L.load().ddst_destroy(ctx)


class Solver:
    """Owning wrapper: setup (factor) -> build_transfer -> [compress] -> solve / solve_adjoint."""

    def __init__(self, problems, precision="mixed", stream=None, **opts):
        if isinstance(problems, dict):
            problems = [problems]
        self.problems = problems
        self.options = ddst_options_default(precision=precision, **opts)
        self._keep = problems  # keep host arrays alive during setup
        self.ctx = ddst_setup_batch(problems, self.options, stream)

    @property
    def precision(self):
        """"fp64" or "mixed" (the choice of precision="auto")."""
        return ddst_get_precision(self.ctx)

    def build_transfer(self):
        ddst_build_transfer(self.ctx)
        return self

    def compress(self, tol):
        ddst_compress(self.ctx, tol)
        return self

    def compress_hbs(self, rank, oversample=10):
        ddst_compress_hbs(self.ctx, rank, oversample)
        return self

    def solve(self, f, g, u, **kw):
        if len(self.problems) == 1:
            _check_sizes(self.problems[0], f=f, g=g, u=u)
        return ddst_solve(self.ctx, f, g, u, **kw)

    def close(self):
        if self.ctx:
            ddst_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    import torch

    class DDSTSolve(torch.autograd.Function):
        """``u = A(a)^{-1} b(f, g)`` on the GPU; backward is the hand-written discrete adjoint.

        forward(a, f, g, spec) with ``spec = dict(dim, n, w, b=(..), c=None, precision=..,
        compress_tol=None)``; the local factors are recomputed for every forward call.
        """

        @staticmethod
        def forward(ctx, a, f, g, spec):
            opts = dict(spec.get("options", {}))
            sol = Solver(dict(dim=spec["dim"], n=spec["n"], w=spec["w"], a=a.detach().contiguous(),
                              b=spec.get("b"), c=spec.get("c")),
                         precision=spec.get("precision", "mixed"), **opts)
            sol.build_transfer()
            if spec.get("compress_tol"):
                sol.compress(spec["compress_tol"])
            u = torch.empty_like(f)
            sol.solve(f.detach().contiguous(), g.detach().contiguous(), u)
            ctx.sol = sol
            ctx.shapes = (a.shape, f.shape, g.shape)
            return u

        @staticmethod
        def backward(ctx, gu):
            sol = ctx.sol
            sa, sf, sg = ctx.shapes
            dev = gu.device
            da = torch.empty(sa, dtype=torch.float64, device=dev)
            df = torch.empty(sf, dtype=torch.float64, device=dev)
            dg = torch.empty(sg, dtype=torch.float64, device=dev)
            ddst_solve_adjoint(sol.ctx, gu.contiguous(), df, dg, da)
            sol.close()
            ctx.sol = None
            return da, df, dg, None

    return DDSTSolve


class _Lazy:
    _cls = None

    def __getattr__(self, item):
        if _Lazy._cls is None:
            _Lazy._cls = _make_autograd()
        return getattr(_Lazy._cls, item)


DDSTSolve = _Lazy()
