"""Python binding of the C ABI in ``include/chem.h`` -- argument marshalling only.

Every computation runs in ``_native/libchemgb.so`` (hand-written sm_103a CUDA).  Device arrays are
torch tensors (float64 / int32, contiguous, on the handle's device); the CUDA stream is torch's current
stream unless one is passed.  There is no CPU path: if the library cannot be built or loaded, or a
call fails, a ``ChemError`` is raised.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

from . import build as _build

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_vp = C.c_void_p


class ChemError(RuntimeError):
    pass


class MechDescC(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int), ("n_elements", C.c_int),
                ("W", _dp), ("nasa_lo", _dp), ("nasa_hi", _dp), ("T_mid", _dp), ("comp", _ip),
                ("reac_ptr", _ip), ("reac_sp", _ip), ("reac_nu", _ip),
                ("prod_ptr", _ip), ("prod_sp", _ip), ("prod_nu", _ip),
                ("A", _dp), ("b", _dp), ("Ea", _dp), ("rtype", _ip), ("reversible", _ip),
                ("eff_ptr", _ip), ("eff_sp", _ip), ("eff_alpha", _dp), ("troe", _dp), ("low", _dp)]


class InfoC(C.Structure):
    _fields_ = [("n_species", C.c_int), ("n_reactions", C.c_int), ("n_state", C.c_int), ("nnz_S", C.c_int),
                ("nnz_LU", C.c_int), ("lu_steps", C.c_int), ("solve_steps", C.c_int),
                ("smem_per_cell", C.c_int), ("n_dslots", C.c_int), ("jac_passes", C.c_int),
                ("smem_adjoint_per_cell", C.c_int), ("max_block_cells", C.c_int * 3),
                ("resident_cells", C.c_int * 3), ("auto_warps_per_cell", C.c_int),
                ("auto_cells_per_warp", C.c_int)]


class OptsC(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("h_init", C.c_double), ("h_min", C.c_double),
                ("time_budget_s", C.c_double), ("max_substeps", C.c_int), ("max_nonfinite", C.c_int),
                ("mode", C.c_int), ("block_cells", C.c_int), ("chunk", C.c_int), ("naccept", _vp),
                ("trace", _vp), ("trace_cap", C.c_int), ("ckpt_every", C.c_int), ("tape_steps", C.c_int),
                ("warps_per_cell", C.c_int), ("method", C.c_int), ("cells_per_warp", C.c_int),
                ("tabulate", C.c_int), ("tab_tol", C.c_double), ("specialized", C.c_int)]


class MapOptsC(C.Structure):
    _fields_ = [("T_max", C.c_double), ("dT", C.c_double), ("n_species", C.c_int), ("species", C.c_int * 8),
                ("dY", C.c_double * 8)]


CELL_STATUS = {0: "OK", 1: "MAXSTEPS", 2: "HMIN", 3: "NONFINITE", 4: "BADINPUT", 5: "TIMEOUT"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "chem.h")

_lib = None


def declared_functions():
    """Names of the functions ``include/chem.h`` declares."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(chem_\w+)\s*\(", text, re.M)))


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.chem_create.argtypes = [C.POINTER(MechDescC), C.c_int, C.POINTER(_vp)]
        L.chem_destroy.argtypes = [_vp]
        L.chem_last_error.restype = C.c_char_p
        L.chem_info.argtypes = [_vp, C.POINTER(InfoC)]
        L.chem_jacobian_pattern.argtypes = [_vp, _ip, _ip]
        L.chem_export_plan.argtypes = [_vp, C.c_int, _ip, _ip]
        L.chem_rates.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.chem_jacobian.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.chem_integrate.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(OptsC), _vp]
        L.chem_integrate_noalloc.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(OptsC),
                                             _vp]
        L.chem_set_params.argtypes = [_vp, _vp, _vp, _vp]
        L.chem_adjoint.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                   C.POINTER(OptsC), _vp]
        L.chem_eval_elementary.argtypes = [C.c_int, C.c_int, _vp, _vp, _vp]
        L.chem_create_from_json.argtypes = [C.c_char_p, C.c_int, C.POINTER(_vp)]
        L.chem_balance_plan.argtypes = [C.c_int, _vp, _vp, _vp]
        L.chem_integrate_mapped.argtypes = [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(OptsC),
                                            C.POINTER(MapOptsC), _vp, C.POINTER(C.c_int), _vp]
        L.chem_specialize.argtypes = [_vp, C.POINTER(C.c_double)]
        L.chem_specialized_source.argtypes = [_vp, C.c_char_p, C.POINTER(C.c_int)]
        for f in ("chem_integrate_mapped", "chem_balance_plan", "chem_eval_elementary", "chem_create_from_json", "chem_create", "chem_destroy", "chem_info", "chem_jacobian_pattern", "chem_export_plan",
                  "chem_rates", "chem_jacobian", "chem_integrate", "chem_integrate_noalloc", "chem_set_params",
                  "chem_adjoint", "chem_specialize", "chem_specialized_source"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().chem_last_error().decode(errors="replace")
        raise ChemError(f"{what} failed (status {rc}): {msg}")


def _dptr(t, dtype, n, name):
    """Device pointer of a contiguous tensor with at least n elements of dtype (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, {n} needed")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Mechanism:
    """A compiled mechanism (``chem_create``).  ``device=-1`` compiles on the host only."""

    def __init__(self, desc, device: int = 0, json_text: Optional[str] = None):
        self.desc = desc
        self.device = device
        if json_text is not None:           # chem_create_from_json: the library parses the text
            h = _vp()
            _check(lib().chem_create_from_json(json_text.encode(), device, C.byref(h)), "chem_create_from_json")
            self._h = h
            self._finish()
            return
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        k = dict(W=f64(desc.W), lo=f64(desc.nasa_lo).ravel(), hi=f64(desc.nasa_hi).ravel(), Tm=f64(desc.T_mid),
                 comp=i32(desc.comp).ravel(), rp=i32(desc.reac_ptr), rs=i32(desc.reac_sp), rn=i32(desc.reac_nu),
                 pp=i32(desc.prod_ptr), ps=i32(desc.prod_sp), pn=i32(desc.prod_nu), A=f64(desc.A), b=f64(desc.b),
                 Ea=f64(desc.Ea), rt=i32(desc.rtype), rev=i32(desc.reversible), ep=i32(desc.eff_ptr),
                 es=i32(desc.eff_sp), ea=f64(desc.eff_alpha), troe=f64(desc.troe).ravel(), low=f64(desc.low).ravel())
        self._keep = k
        d = lambda a: a.ctypes.data_as(_dp)
        i = lambda a: a.ctypes.data_as(_ip)
        n_el = int(np.asarray(desc.comp).shape[1]) if np.asarray(desc.comp).ndim == 2 else 0
        self._desc = MechDescC(int(len(desc.W)), int(len(desc.A)), n_el, d(k["W"]), d(k["lo"]), d(k["hi"]), d(k["Tm"]),
                               i(k["comp"]) if n_el else None, i(k["rp"]), i(k["rs"]), i(k["rn"]), i(k["pp"]),
                               i(k["ps"]), i(k["pn"]), d(k["A"]), d(k["b"]), d(k["Ea"]), i(k["rt"]), i(k["rev"]),
                               i(k["ep"]), i(k["es"]), d(k["ea"]), d(k["troe"]), d(k["low"]))
        h = _vp()
        _check(lib().chem_create(C.byref(self._desc), device, C.byref(h)), "chem_create")
        self._h = h
        self._finish()

    def _finish(self):
        self.info = self._info()
        self.n = self.info["n_species"]
        self.R = self.info["n_reactions"]
        self.m = self.info["n_state"]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().chem_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _info(self):
        inf = InfoC()
        _check(lib().chem_info(self._h, C.byref(inf)), "chem_info")
        out = {}
        for f, _ in InfoC._fields_:
            v = getattr(inf, f)
            out[f] = list(v) if hasattr(v, "__len__") else v
        return out

    def jacobian_pattern(self):
        m, nnz = self.info["n_state"], self.info["nnz_S"]
        rp = np.zeros(m + 1, dtype=np.int32)
        ci = np.zeros(nnz, dtype=np.int32)
        _check(lib().chem_jacobian_pattern(self._h, rp.ctypes.data_as(_ip), ci.ctypes.data_as(_ip)),
               "chem_jacobian_pattern")
        return rp, ci

    def export_plan(self, which: int) -> np.ndarray:
        cnt = C.c_int(0)
        _check(lib().chem_export_plan(self._h, which, None, C.byref(cnt)), "chem_export_plan")
        out = np.zeros(max(cnt.value, 1), dtype=np.int32)
        _check(lib().chem_export_plan(self._h, which, out.ctypes.data_as(_ip), C.byref(cnt)), "chem_export_plan")
        return out[: cnt.value]

    def specialize(self) -> float:
        """chem_specialize: compile (or load from the cache) the mechanism-specialised one-warp kernels for
        this handle; returns the compile time in seconds (0 from the cache)."""
        t = C.c_double(0.0)
        _check(lib().chem_specialize(self._h, C.byref(t)), "chem_specialize")
        return t.value

    def specialized_source(self) -> str:
        """chem_specialized_source: the run-time compiled source of ``specialize``."""
        n = C.c_int(0)
        _check(lib().chem_specialized_source(self._h, None, C.byref(n)), "chem_specialized_source")
        buf = C.create_string_buffer(n.value)
        _check(lib().chem_specialized_source(self._h, buf, C.byref(n)), "chem_specialized_source")
        return buf.value.decode()

    # ---------------------------------------------------------------------------------- compute
    def rates(self, T, p, Y, dTdt, dYdt, wdot=None, stream=None):
        """chem_rates on device tensors (outputs written in place)."""
        import torch
        N = T.numel()
        n = self.n
        _check(lib().chem_rates(self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
                                _dptr(Y, torch.float64, n * N, "Y"), _dptr(dTdt, torch.float64, N, "dTdt"),
                                _dptr(dYdt, torch.float64, n * N, "dYdt"), _dptr(wdot, torch.float64, n * N, "wdot"),
                                _stream(stream)), "chem_rates")

    def jacobian(self, T, p, Y, S_vals, u, v, stream=None):
        """chem_jacobian on device tensors (outputs written in place)."""
        import torch
        N = T.numel()
        _check(lib().chem_jacobian(self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
                                   _dptr(Y, torch.float64, self.n * N, "Y"),
                                   _dptr(S_vals, torch.float64, self.info["nnz_S"] * N, "S_vals"),
                                   _dptr(u, torch.float64, self.m * N, "u"), _dptr(v, torch.float64, self.m * N, "v"),
                                   _stream(stream)), "chem_jacobian")

    def integrate(self, T, p, Y, dt, h_io, nsub, status, rtol=1e-6, atol=1e-12, h_init=0.0, h_min=0.0,
                  time_budget_s=0.0, max_substeps=0, max_nonfinite=0, mode=0, block_cells=0, chunk=0, naccept=None,
                  trace=None, warps_per_cell=0, method=0, cells_per_warp=0, tabulate=0, tab_tol=0.0, specialized=0,
                  stream=None):
        """chem_integrate on device tensors: T, Y, h_io, nsub, status (and naccept) are updated in place.
        specialized=1 runs the kernels ``specialize()`` compiled for this mechanism."""
        import torch
        N = T.numel()
        cap = trace.numel() // max(N, 1) if trace is not None else 0
        o = OptsC(rtol, atol, h_init, h_min, time_budget_s, max_substeps, max_nonfinite, mode, block_cells, chunk,
                  _dptr(naccept, torch.int32, N, "naccept"), _dptr(trace, torch.float64, cap * N, "trace"), cap,
                  0, 0, warps_per_cell, method, cells_per_warp, tabulate, tab_tol, specialized)
        _check(lib().chem_integrate(self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
                                    _dptr(Y, torch.float64, self.n * N, "Y"), _dptr(dt, torch.float64, N, "dt"),
                                    _dptr(h_io, torch.float64, N, "h_io"), _dptr(nsub, torch.int32, N, "nsub"),
                                    _dptr(status, torch.int32, N, "status"), C.byref(o), _stream(stream)),
               "chem_integrate")


    def set_params(self, dlnA=None, dEa=None, stream=None):
        """chem_set_params: shift ln A and Ea of every reaction (device tensors [R], description order)."""
        import torch
        _check(lib().chem_set_params(self._h, _dptr(dlnA, torch.float64, self.R, "dlnA"),
                                     _dptr(dEa, torch.float64, self.R, "dEa"), _stream(stream)), "chem_set_params")

    def adjoint(self, T, p, Y, dt, gT, gY, grad_lnA, grad_Ea, status, grad_cell=None, gT0=None, gY0=None, rtol=1e-6,
                atol=1e-12, h_init=0.0, h_min=0.0, max_substeps=0, max_nonfinite=0, ckpt_every=0, tape_steps=0,
                stream=None):
        """chem_adjoint on device tensors: T, Y in/out (initial -> final state); gradients written in place."""
        import torch
        N = T.numel()
        o = OptsC(rtol, atol, h_init, h_min, 0.0, max_substeps, max_nonfinite, 0, 0, 0, None, None, 0, ckpt_every,
                  tape_steps)
        _check(lib().chem_adjoint(
            self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
            _dptr(Y, torch.float64, self.n * N, "Y"), _dptr(dt, torch.float64, N, "dt"),
            _dptr(gT, torch.float64, N, "gT"), _dptr(gY, torch.float64, self.n * N, "gY"),
            _dptr(grad_lnA, torch.float64, self.R, "grad_lnA"), _dptr(grad_Ea, torch.float64, self.R, "grad_Ea"),
            _dptr(grad_cell, torch.float64, 2 * self.R * N, "grad_cell"), _dptr(gT0, torch.float64, N, "gT0"),
            _dptr(gY0, torch.float64, self.n * N, "gY0"), _dptr(status, torch.int32, N, "status"), C.byref(o),
            _stream(stream)), "chem_adjoint")

    def integrate_noalloc(self, T, p, Y, dt, h_io, nsub, status, rtol=1e-6, atol=1e-12, h_init=0.0, h_min=0.0,
                          time_budget_s=0.0, max_substeps=0, max_nonfinite=0, block_cells=0, chunk=0, naccept=None,
                          trace=None, warps_per_cell=0, method=0, cells_per_warp=0, tabulate=0, tab_tol=0.0,
                          specialized=0, stream=None):
        """chem_integrate_noalloc: the sorted work-queue integration with its scratch in the library's
        static device memory (no allocation in the call; at most 1,048,576 cells; calls must not overlap
        on the GPU).  In-place like ``integrate``."""
        import torch
        N = T.numel()
        cap = trace.numel() // max(N, 1) if trace is not None else 0
        o = OptsC(rtol, atol, h_init, h_min, time_budget_s, max_substeps, max_nonfinite, 1, block_cells, chunk,
                  _dptr(naccept, torch.int32, N, "naccept"), _dptr(trace, torch.float64, cap * N, "trace"), cap,
                  0, 0, warps_per_cell, method, cells_per_warp, tabulate, tab_tol, specialized)
        _check(lib().chem_integrate_noalloc(
            self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
            _dptr(Y, torch.float64, self.n * N, "Y"), _dptr(dt, torch.float64, N, "dt"),
            _dptr(h_io, torch.float64, N, "h_io"), _dptr(nsub, torch.int32, N, "nsub"),
            _dptr(status, torch.int32, N, "status"), C.byref(o), _stream(stream)), "chem_integrate_noalloc")


    def integrate_mapped(self, T, p, Y, dt, h_io, nsub, status, ref, mapping=None, rtol=1e-6, atol=1e-12,
                         h_init=0.0, h_min=0.0, max_substeps=0, max_nonfinite=0, mode=0, block_cells=0, chunk=0,
                         warps_per_cell=0, method=0, cells_per_warp=0, tabulate=0, tab_tol=0.0,
                         stream=None) -> int:
        """chem_integrate_mapped: like `integrate`, with zonal reference-cell mapping.  mapping: None or
        dict(T_max, dT, species=[...], dY=[...]).  ref (int32 [N], device) receives each cell's reference.
        Returns the number of cells integrated."""
        import torch
        N = T.numel()
        o = OptsC(rtol, atol, h_init, h_min, 0.0, max_substeps, max_nonfinite, mode, block_cells, chunk, None, None,
                  0, 0, 0, warps_per_cell, method, cells_per_warp, tabulate, tab_tol)
        mp = None
        if mapping is not None:
            sp = list(mapping.get("species", ()))
            dy = list(mapping.get("dY", ()))
            if len(sp) != len(dy) or len(sp) > 8:
                raise ValueError("mapping: species and dY must have the same length, at most 8")
            mp = MapOptsC(float(mapping["T_max"]), float(mapping["dT"]), len(sp), (C.c_int * 8)(*sp),
                          (C.c_double * 8)(*dy))
        cnt = C.c_int(0)
        _check(lib().chem_integrate_mapped(
            self._h, N, _dptr(T, torch.float64, N, "T"), _dptr(p, torch.float64, N, "p"),
            _dptr(Y, torch.float64, self.n * N, "Y"), _dptr(dt, torch.float64, N, "dt"),
            _dptr(h_io, torch.float64, N, "h_io"), _dptr(nsub, torch.int32, N, "nsub"),
            _dptr(status, torch.int32, N, "status"), C.byref(o), C.byref(mp) if mp is not None else None,
            _dptr(ref, torch.int32, N, "ref"), C.byref(cnt), _stream(stream)), "chem_integrate_mapped")
        return int(cnt.value)


def eval_elementary(fn: int, x, y, stream=None):
    """chem_eval_elementary: y = f(x) on the device (fn 0 library exp, 1 CUDA exp, 2 library log,
    3 CUDA log)."""
    import torch
    N = x.numel()
    _check(lib().chem_eval_elementary(fn, N, _dptr(x, torch.float64, N, "x"), _dptr(y, torch.float64, N, "y"),
                                      _stream(stream)), "chem_eval_elementary")


def create(desc, device: int = 0) -> Mechanism:
    """chem_create."""
    return Mechanism(desc, device)


def create_from_json(json_text: str, device: int = 0) -> Mechanism:
    """chem_create_from_json: the library parses the text.  ``desc`` is then the Python reading of the same
    text when it carries the generator's metadata too (used by host-side helpers such as the autotuner's
    cache key), else None."""
    from . import synth
    h = Mechanism(None, device, json_text=json_text)
    try:
        h.desc = synth.MechDesc.from_json(json_text)
    except (KeyError, TypeError, ValueError):
        h.desc = None
    return h


def balance_plan(counts, costs) -> np.ndarray:
    """chem_balance_plan: destination rank of every cell.  counts[r] = cells of rank r; costs = all ranks'
    per-cell costs, rank 0's first, each rank's in local order.  Host arrays."""
    cnt = np.ascontiguousarray(counts, dtype=np.int64)
    cst = np.ascontiguousarray(costs, dtype=np.float64)
    if cst.shape[0] != int(cnt.sum()):
        raise ValueError("costs must hold sum(counts) values")
    dest = np.empty(cst.shape[0], dtype=np.int32)
    _check(lib().chem_balance_plan(len(cnt), cnt.ctypes.data_as(_vp), cst.ctypes.data_as(_vp),
                                   dest.ctypes.data_as(_vp)), "chem_balance_plan")
    return dest
