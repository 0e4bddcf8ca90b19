"""PyTorch-facing API over the C ABI (device memory and streams come from torch;
every step of the computation runs in libconvgb.so kernels).

Profile tensors are level-major ``[pver, ld]`` (columns innermost, the layout of
include/conv.h); column tensors are ``[ld]``.  ``ld`` may exceed the number of
columns processed (``n_cols``).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

_OUT_FIELDS = ("dTdt", "dqdt", "prec", "flags", "kb", "klcl", "ktop", "kaux", "cape", "mb",
               "cons_err", "mu", "du", "md")
_FLUX_FIELDS = ("mu", "du", "md")
_PREC = {"fp64": L.CONV_FP64, "mixed": L.CONV_MIXED}
_PATH = {"auto": L.CONV_PATH_AUTO, "plain": L.CONV_PATH_PLAIN, "compact": L.CONV_PATH_COMPACT}


def real_dtype(precision: str) -> torch.dtype:
    return torch.float64 if precision == "fp64" else torch.float32


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _require_cuda(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def new_outputs(pver: int, ld: int, precision: str, device="cuda", flux: bool = False) -> dict:
    """Allocate one scheme's output tensors; flux=True adds the mass-flux
    profiles mu, du, md that tracer_transport needs."""
    rd = real_dtype(precision)
    f64, i32 = torch.float64, torch.int32
    extra = {k: torch.empty((pver, ld), dtype=rd, device=device) for k in _FLUX_FIELDS} \
        if flux else {}
    return dict(**extra, dTdt=torch.empty((pver, ld), dtype=rd, device=device),
                dqdt=torch.empty((pver, ld), dtype=rd, device=device),
                prec=torch.empty(ld, dtype=f64, device=device),
                flags=torch.empty(ld, dtype=i32, device=device),
                kb=torch.empty(ld, dtype=i32, device=device),
                klcl=torch.empty(ld, dtype=i32, device=device),
                ktop=torch.empty(ld, dtype=i32, device=device),
                kaux=torch.empty(ld, dtype=i32, device=device),
                cape=torch.empty(ld, dtype=f64, device=device),
                mb=torch.empty(ld, dtype=f64, device=device),
                cons_err=torch.empty(ld, dtype=f64, device=device))


def _out_struct(o: dict, pver: int, ld: int, precision: str) -> L.Out:
    rd = real_dtype(precision)
    for k in ("dTdt", "dqdt"):
        _require_cuda(o[k], k, rd, (pver, ld))
    for k in ("prec", "cape", "mb", "cons_err"):
        if o.get(k) is not None:
            _require_cuda(o[k], k, torch.float64, (ld,))
    for k in ("flags", "kb", "klcl", "ktop", "kaux"):
        if o.get(k) is not None:
            _require_cuda(o[k], k, torch.int32, (ld,))
    for k in _FLUX_FIELDS:
        if o.get(k) is not None:
            _require_cuda(o[k], k, rd, (pver, ld))
    return L.Out(*[_ptr(o.get(k)) for k in _OUT_FIELDS])


class VerticalGrid:
    """Hybrid interface coefficients (host arrays of pver+1 doubles) and p0."""

    def __init__(self, hyai, hybi, p0: float = 1.0e5):
        self.hyai = np.ascontiguousarray(hyai, dtype=np.float64)
        self.hybi = np.ascontiguousarray(hybi, dtype=np.float64)
        if self.hyai.shape != self.hybi.shape or self.hyai.ndim != 1:
            raise ValueError("hyai/hybi must be 1-D of equal length")
        self.pver = self.hyai.shape[0] - 1
        self.p0 = float(p0)

    def struct(self, n_cols: int, ld: int) -> L.Grid:
        dp = C.POINTER(C.c_double)
        return L.Grid(self.pver, int(n_cols), int(ld), 0, self.hyai.ctypes.data_as(dp),
                      self.hybi.ctypes.data_as(dp), self.p0)


_MAP = {"auto": L.CONV_MAP_DEFAULT, "thread": L.CONV_MAP_THREAD, "warp": L.CONV_MAP_WARP}


def _launch(path: str, block_threads: int = 0, stage_events=None,
            mapping: str = "auto") -> L.Launch:
    if mapping not in _MAP:
        raise ValueError(f"mapping must be one of {list(_MAP)}")
    lc = L.Launch(_PATH[path], int(block_threads), _MAP[mapping], 0, None)
    if stage_events is not None:
        if len(stage_events) != 3:
            raise ValueError("stage_events needs three torch.cuda.Event")
        handles = []
        for ev in stage_events:
            if ev.cuda_event == 0:  # torch creates the CUDA event lazily
                ev.record()
            handles.append(ev.cuda_event)
        arr = (C.c_void_p * 3)(*handles)
        lc._keep = arr
        lc.stage_events = C.cast(arr, C.POINTER(C.c_void_p))
    return lc


def workspace_bytes(vgrid: VerticalGrid, n_cols: int, ld: int, precision="fp64",
                    path="plain") -> int:
    g = vgrid.struct(n_cols, ld)
    lc = _launch(path)
    return int(L.lib().conv_workspace_bytes(C.byref(g), _PREC[precision], C.byref(lc)))


class Workspace:
    """Caller-owned device workspace, grown on demand (allocation happens here, in
    torch, never inside the library's run calls)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes: int):
        if nbytes == 0:
            return None, 0
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.buf.data_ptr()
        off = (-base) % 256
        return C.c_void_p(base + off), self.buf.numel() - off


_default_ws = {}


def _ws_for(device, ws: Workspace | None):
    if ws is not None:
        return ws
    key = str(device)
    if key not in _default_ws:
        _default_ws[key] = Workspace(device)
    return _default_ws[key]


def _common(T, q, ps, vgrid, n_cols, precision, lam, tau):
    if precision not in _PREC:
        raise ValueError(f"precision must be one of {list(_PREC)}")
    rd = real_dtype(precision)
    if T.dim() != 2:
        raise ValueError("T must be [pver, ld]")
    pver, ld = T.shape
    if pver != vgrid.pver:
        raise ValueError(f"T has {pver} levels, vertical grid has {vgrid.pver}")
    _require_cuda(T, "T", rd, (pver, ld))
    _require_cuda(q, "q", rd, (pver, ld))
    _require_cuda(ps, "ps", torch.float64, (ld,))
    for name, t in (("lam", lam), ("tau", tau)):
        if t is not None:
            _require_cuda(t, name, torch.float64, (ld,))
    n = ld if n_cols is None else int(n_cols)
    inp = L.In(_ptr(T), _ptr(q), _ptr(ps), _ptr(lam), _ptr(tau))
    return pver, ld, n, inp


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _shift(struct, col0: int, sizes: dict):
    """Offset the column pointers of a conv_in / conv_out struct by col0 columns
    (element sizes by field); the leading dimension stays that of the arrays."""
    for name, size in sizes.items():
        v = getattr(struct, name)
        if v:
            setattr(struct, name, v + col0 * size)
    return struct


def _in_sizes(precision):
    rb = 8 if precision == "fp64" else 4
    return {"T": rb, "q": rb, "ps": 8, "lam": 8, "tau": 8}


def _out_sizes(precision):
    rb = 8 if precision == "fp64" else 4
    d = {k: rb for k in ("dTdt", "dqdt", "mu", "du", "md")}
    d.update({k: 8 for k in ("prec", "cape", "mb", "cons_err")})
    d.update({k: 4 for k in ("flags", "kb", "klcl", "ktop", "kaux")})
    return d


def deep_shallow(T, q, ps, vgrid: VerticalGrid, *, dt: float = 1800.0, precision="fp64",
                 lam=None, tau=None, deep_params=None, shallow_params=None, path="auto",
                 block_threads=0, n_cols=None, out_deep=None, out_shallow=None,
                 workspace: Workspace | None = None, stream=None, stage_events=None,
                 col0: int = 0, mapping: str = "auto"):
    """Deep then shallow convection (Alg. 1 order) in one fused call.

    Returns ``(deep_out, shallow_out)`` dicts of output tensors.  stage_events:
    optional three torch.cuda.Event the library records around its passes.
    col0: first column of the range processed (columns col0 .. col0 + n_cols - 1
    of every [pver, ld] / [ld] tensor; n_cols defaults to the rest of ld); the
    other columns of the outputs are left untouched.  mapping: the compacted
    trigger pass's mapping, "thread" (one column per thread, the default for
    "auto") or "warp" (one column per warp, lane k = level k)."""
    pver, ld, n, inp = _common(T, q, ps, vgrid, n_cols, precision, lam, tau)
    col0 = int(col0)
    if n_cols is None:
        n = ld - col0
    if col0 < 0 or n < 0 or col0 + n > ld:
        raise ValueError(f"columns {col0}..{col0 + n - 1} outside ld = {ld}")
    od = out_deep if out_deep is not None else new_outputs(pver, ld, precision, T.device)
    os_ = out_shallow if out_shallow is not None else new_outputs(pver, ld, precision, T.device)
    dp = deep_params or L.deep_defaults()
    sp = shallow_params or L.shallow_defaults()
    g = vgrid.struct(n, ld)
    lc = _launch(path, block_threads, stage_events, mapping)
    nb = int(L.lib().conv_workspace_bytes(C.byref(g), _PREC[precision], C.byref(lc)))
    wp, wn = _ws_for(T.device, workspace).get(nb)
    so_d = _out_struct(od, pver, ld, precision)
    so_s = _out_struct(os_, pver, ld, precision)
    if col0:
        _shift(inp, col0, _in_sizes(precision))
        _shift(so_d, col0, _out_sizes(precision))
        _shift(so_s, col0, _out_sizes(precision))
    st = L.lib().conv_deep_shallow_run(
        C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp), float(dt), _PREC[precision],
        C.byref(so_d), C.byref(so_s), C.byref(lc), wp, wn, _stream(stream))
    L.check(st, "conv_deep_shallow_run")
    return od, os_


class PreparedStep:
    """The fused deep -> shallow step with its C-ABI arguments marshalled once,
    for launch-bound loops: each call is one library call (the library records
    the optional stage events and launches its kernels), with no Python
    validation or struct building on the way.  The tensors given here must stay
    alive and in place while the object is used."""

    def __init__(self, T, q, ps, vgrid: VerticalGrid, *, dt: float = 1800.0,
                 precision="fp64", lam=None, tau=None, deep_params=None, shallow_params=None,
                 path="auto", block_threads=0, n_cols=None, out_deep=None, out_shallow=None,
                 workspace: Workspace | None = None, stream=None, mapping: str = "auto"):
        pver, ld, n, self._inp = _common(T, q, ps, vgrid, n_cols, precision, lam, tau)
        self.out_deep = out_deep if out_deep is not None else new_outputs(pver, ld, precision,
                                                                          T.device)
        self.out_shallow = out_shallow if out_shallow is not None else new_outputs(
            pver, ld, precision, T.device)
        self._keep = (T, q, ps, lam, tau)
        self._dp = deep_params or L.deep_defaults()
        self._sp = shallow_params or L.shallow_defaults()
        self._g = vgrid.struct(n, ld)
        self._path, self._block, self._mapping = path, int(block_threads), mapping
        lc = _launch(path, block_threads, mapping=mapping)
        nb = int(L.lib().conv_workspace_bytes(C.byref(self._g), _PREC[precision], C.byref(lc)))
        self._ws = _ws_for(T.device, workspace)
        self._wp, self._wn = self._ws.get(nb)
        self._od = _out_struct(self.out_deep, pver, ld, precision)
        self._os = _out_struct(self.out_shallow, pver, ld, precision)
        self._args = (C.byref(self._g), C.byref(self._inp), C.byref(self._dp),
                      C.byref(self._sp), float(dt), _PREC[precision], C.byref(self._od),
                      C.byref(self._os))
        self._tail = (self._wp, self._wn, _stream(stream))
        self._lc = lc
        self._fn = L.lib().conv_deep_shallow_run

    def launch_struct(self, stage_events=None) -> L.Launch:
        """A launch descriptor with stage events, to build outside a timed loop."""
        return _launch(self._path, self._block, stage_events, self._mapping)

    def __call__(self, launch: L.Launch | None = None):
        st = self._fn(*self._args, C.byref(launch if launch is not None else self._lc),
                      *self._tail)
        if st != L.CONV_OK:
            L.check(st, "conv_deep_shallow_run")
        return self.out_deep, self.out_shallow


def tracer_transport(tracers, ps, vgrid: VerticalGrid, *, deep_out=None, shallow_out=None,
                     dt: float = 1800.0, precision="fp64", n_cols=None, tend_deep=None,
                     tend_shallow=None, stream=None):
    """Convective transport of passive tracers ([ntr][pver][ld] tensor) by the
    plumes of a run whose outputs hold the mass-flux profiles (new_outputs(...,
    flux=True)).  Returns (tend_deep, tend_shallow) (None for a scheme not
    given); with both schemes the shallow one transports the deep-updated
    tracer max(c + dt tend_deep, 0)."""
    rd = real_dtype(precision)
    if tracers.dim() != 3 or not tracers.is_cuda or tracers.dtype != rd or \
            not tracers.is_contiguous():
        raise TypeError(f"tracers must be a contiguous CUDA {rd} tensor [ntr][pver][ld]")
    ntr, pver, ld = tracers.shape
    if pver != vgrid.pver:
        raise ValueError(f"tracers have {pver} levels, the grid {vgrid.pver}")
    n = ld if n_cols is None else int(n_cols)
    _require_cuda(ps, "ps", torch.float64, (ld,))
    if deep_out is None and shallow_out is None:
        raise ValueError("give deep_out and/or shallow_out")
    outs = []
    for o, t in ((deep_out, tend_deep), (shallow_out, tend_shallow)):
        if o is None:
            outs.append((None, None))
            continue
        if t is None:
            t = torch.empty_like(tracers)
        elif t.shape != tracers.shape or t.dtype != rd or not t.is_cuda or not t.is_contiguous():
            raise TypeError("tendency tensors must match the tracers")
        outs.append((_out_struct(o, pver, ld, precision), t))
    g = vgrid.struct(n, ld)
    (od, td), (os_, ts) = outs
    st = L.lib().conv_tracer_transport(
        C.byref(g), _ptr(ps), None if od is None else C.byref(od),
        None if os_ is None else C.byref(os_), float(dt), int(ntr), _ptr(tracers), _ptr(td),
        _ptr(ts), _PREC[precision], _stream(stream))
    L.check(st, "conv_tracer_transport")
    return td, ts


def momentum_transport(uv, ps, vgrid: VerticalGrid, *, deep_out=None, shallow_out=None,
                       dt: float = 1800.0, precision="fp64", cp_up: float = 0.7,
                       cp_down: float = 0.7, n_cols=None, tend_deep=None, tend_shallow=None,
                       stream=None):
    """Convective momentum transport of the wind components uv ([2][pver][ld]
    tensor, u then v) by the plumes of a run whose outputs hold the mass-flux
    profiles (new_outputs(..., flux=True)), with the plumes' pressure-gradient
    coefficients cp_up (updrafts) and cp_down (downdraft).  Returns (tend_deep,
    tend_shallow) (None for a scheme not given); with both schemes the shallow
    one transports the deep-updated wind u + dt tend_deep."""
    rd = real_dtype(precision)
    if uv.dim() != 3 or uv.shape[0] != 2 or not uv.is_cuda or uv.dtype != rd or \
            not uv.is_contiguous():
        raise TypeError(f"uv must be a contiguous CUDA {rd} tensor [2][pver][ld]")
    _, pver, ld = uv.shape
    if pver != vgrid.pver:
        raise ValueError(f"uv has {pver} levels, the grid {vgrid.pver}")
    n = ld if n_cols is None else int(n_cols)
    _require_cuda(ps, "ps", torch.float64, (ld,))
    if deep_out is None and shallow_out is None:
        raise ValueError("give deep_out and/or shallow_out")
    outs = []
    for o, t in ((deep_out, tend_deep), (shallow_out, tend_shallow)):
        if o is None:
            outs.append((None, None))
            continue
        if t is None:
            t = torch.empty_like(uv)
        elif t.shape != uv.shape or t.dtype != rd or not t.is_cuda or not t.is_contiguous():
            raise TypeError("tendency tensors must match uv")
        outs.append((_out_struct(o, pver, ld, precision), t))
    g = vgrid.struct(n, ld)
    (od, td), (os_, ts) = outs
    st = L.lib().conv_momentum_transport(
        C.byref(g), _ptr(ps), None if od is None else C.byref(od),
        None if os_ is None else C.byref(os_), float(dt), float(cp_up), float(cp_down), _ptr(uv),
        _ptr(td), _ptr(ts), _PREC[precision], _stream(stream))
    L.check(st, "conv_momentum_transport")
    return td, ts


def deep_shallow_tracers(T, q, ps, tracers, vgrid: VerticalGrid, *, dt: float = 1800.0,
                         precision="fp64", lam=None, tau=None, deep_params=None,
                         shallow_params=None, path="auto", n_cols=None, out_deep=None,
                         out_shallow=None, workspace: Workspace | None = None, stream=None):
    """The fused step with tracers: deep then shallow convection writing their
    mass-flux profiles, then the transport of every tracer by both schemes.
    Returns (deep_out, shallow_out, tend_deep, tend_shallow)."""
    pver, ld = T.shape
    od = out_deep if out_deep is not None else new_outputs(pver, ld, precision, T.device, True)
    os_ = out_shallow if out_shallow is not None else new_outputs(pver, ld, precision,
                                                                   T.device, True)
    deep_shallow(T, q, ps, vgrid, dt=dt, precision=precision, lam=lam, tau=tau,
                 deep_params=deep_params, shallow_params=shallow_params, path=path,
                 n_cols=n_cols, out_deep=od, out_shallow=os_, workspace=workspace, stream=stream)
    td, ts = tracer_transport(tracers, ps, vgrid, deep_out=od, shallow_out=os_, dt=dt,
                              precision=precision, n_cols=n_cols, stream=stream)
    return od, os_, td, ts


def deep(T, q, ps, vgrid: VerticalGrid, *, dt: float = 1800.0, precision="fp64", lam=None,
         tau=None, params=None, path="auto", block_threads=0, n_cols=None, out=None,
         workspace: Workspace | None = None, stream=None):
    """Deep convection only (Alg. 2)."""
    pver, ld, n, inp = _common(T, q, ps, vgrid, n_cols, precision, lam, tau)
    o = out if out is not None else new_outputs(pver, ld, precision, T.device)
    dp = params or L.deep_defaults()
    g = vgrid.struct(n, ld)
    lc = _launch(path, block_threads)
    nb = int(L.lib().conv_workspace_bytes(C.byref(g), _PREC[precision], C.byref(lc)))
    wp, wn = _ws_for(T.device, workspace).get(nb)
    st = L.lib().conv_deep_run(C.byref(g), C.byref(inp), C.byref(dp), float(dt),
                               _PREC[precision], C.byref(_out_struct(o, pver, ld, precision)),
                               C.byref(lc), wp, wn, _stream(stream))
    L.check(st, "conv_deep_run")
    return o


def shallow(T, q, ps, vgrid: VerticalGrid, *, precision="fp64", params=None, path="plain",
            block_threads=0, n_cols=None, out=None, workspace: Workspace | None = None,
            stream=None):
    """Shallow convection only (Alg. 3) on the given state."""
    pver, ld, n, inp = _common(T, q, ps, vgrid, n_cols, precision, None, None)
    o = out if out is not None else new_outputs(pver, ld, precision, T.device)
    sp = params or L.shallow_defaults()
    g = vgrid.struct(n, ld)
    lc = _launch(path, block_threads)
    nb = int(L.lib().conv_workspace_bytes(C.byref(g), _PREC[precision], C.byref(lc)))
    wp, wn = _ws_for(T.device, workspace).get(nb)
    st = L.lib().conv_shallow_run(C.byref(g), C.byref(inp), C.byref(sp), _PREC[precision],
                                  C.byref(_out_struct(o, pver, ld, precision)), C.byref(lc),
                                  wp, wn, _stream(stream))
    L.check(st, "conv_shallow_run")
    return o


class Batch:
    """A batched ensemble: many fused deep->shallow problems (uneven column and
    level counts) run as one trigger launch and one persistent plume launch.

    members: list of dicts with keys T, q, ps (device tensors, [pver, ld] /
    [ld]), vgrid (VerticalGrid), optional lam, tau, n_cols, dt, deep_params,
    shallow_params; outputs are allocated here (``self.outputs[m] = (deep,
    shallow)``) unless given as ``out_deep`` / ``out_shallow``."""

    def __init__(self, members, precision="fp64", device="cuda"):
        self.precision = precision
        self.outputs = []
        self._keep = []
        arr = (L.Member * len(members))()
        for m, mb in enumerate(members):
            T, q, ps, vg = mb["T"], mb["q"], mb["ps"], mb["vgrid"]
            lam, tau = mb.get("lam"), mb.get("tau")
            pver, ld, n, inp = _common(T, q, ps, vg, mb.get("n_cols"), precision, lam, tau)
            od = mb.get("out_deep") or new_outputs(pver, ld, precision, T.device)
            os_ = mb.get("out_shallow") or new_outputs(pver, ld, precision, T.device)
            self.outputs.append((od, os_))
            self._keep.append((T, q, ps, lam, tau, vg))
            arr[m].grid = vg.struct(n, ld)
            arr[m].in_ = inp
            arr[m].deep_out = _out_struct(od, pver, ld, precision)
            arr[m].shallow_out = _out_struct(os_, pver, ld, precision)
            arr[m].deep = mb.get("deep_params") or L.deep_defaults()
            arr[m].shallow = mb.get("shallow_params") or L.shallow_defaults()
            arr[m].dt = float(mb.get("dt", 1800.0))
        h = C.c_void_p()
        L.check(L.lib().conv_batch_plan(arr, len(members), _PREC[precision], C.byref(h)),
                "conv_batch_plan")
        self._h = h
        self.ws = Workspace(device)

    def workspace_bytes(self) -> int:
        return int(L.lib().conv_batch_workspace_bytes(self._h))

    def run(self, stream=None, stage_events=None):
        wp, wn = self.ws.get(self.workspace_bytes())
        ev = None
        if stage_events is not None:
            lc = _launch("auto", 0, stage_events)
            ev = lc.stage_events
            self._ev_keep = lc
        L.check(L.lib().conv_batch_run(self._h, wp, wn, _stream(stream), ev), "conv_batch_run")
        return self.outputs

    def autotune(self, reps: int = 3, stream=None):
        wp, wn = self.ws.get(self.workspace_bytes())
        L.check(L.lib().conv_batch_autotune(self._h, wp, wn, _stream(stream), int(reps)),
                "conv_batch_autotune")
        return self.config()

    def config(self):
        a, b, c, m = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        L.check(L.lib().conv_batch_config(self._h, C.byref(a), C.byref(b), C.byref(c),
                                          C.byref(m)), "conv_batch_config")
        return {"trigger_mapping": "warp" if m.value == L.CONV_MAP_WARP else "thread",
                "trigger_block": a.value, "plume_block": b.value, "plume_grid": c.value}

    def set_config(self, trigger_mapping="thread", trigger_block=128, plume_block=128):
        """Choose the launch shape by hand (see conv_batch_set_config)."""
        m = {"thread": L.CONV_MAP_THREAD, "warp": L.CONV_MAP_WARP}[trigger_mapping]
        L.check(L.lib().conv_batch_set_config(self._h, m, int(trigger_block), int(plume_block)),
                "conv_batch_set_config")
        return self.config()

    def tune_record(self):
        """The last autotune's ms per run of each candidate shape."""
        ms = (C.c_float * 7)()
        L.check(L.lib().conv_batch_tune_record(self._h, ms), "conv_batch_tune_record")
        v = list(ms)
        return {"trigger_thread_block_64": v[0], "trigger_thread_block_128": v[1],
                "trigger_thread_block_256": v[2], "trigger_warp_per_column": v[3],
                "plume_block_64": v[4], "plume_block_128": v[5], "plume_block_256": v[6]}

    def close(self):
        if getattr(self, "_h", None):
            L.lib().conv_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def deep_adjoint(T, q, ps, vgrid: VerticalGrid, *, gP=None, gH=None, w_heat=None,
                 dt: float = 1800.0, lam=None, tau=None, params=None, n_cols=None,
                 gradient=True, objective=False, stream=None):
    """Deep-scheme objective and/or adjoint (FP64, conv_deep_adjoint).

    Per column: P (precipitation) and H = sum_k w_k m_k cp dTdt_k, and the
    gradient of J = gP P + gH H w.r.t. T, q ([pver, ld]), lambda and tau ([ld]).
    w_heat: host sequence of pver weights, None for p_mid/ps.  Returns a dict
    with gT, gq, glambda, gtau (if ``gradient``) and P, H (if ``objective``)."""
    if not (gradient or objective):
        raise ValueError("nothing requested")
    pver, ld, n, inp = _common(T, q, ps, vgrid, n_cols, "fp64", lam, tau)
    f64 = torch.float64
    for name, t in (("gP", gP), ("gH", gH)):
        if t is not None:
            _require_cuda(t, name, f64, (ld,))
    w = None
    if w_heat is not None:
        wa = np.ascontiguousarray(w_heat, dtype=np.float64)
        if wa.shape != (pver,):
            raise ValueError(f"w_heat must have {pver} entries")
        w = wa.ctypes.data_as(C.POINTER(C.c_double))
    res = {}
    if gradient:
        res = dict(gT=torch.empty((pver, ld), dtype=f64, device=T.device),
                   gq=torch.empty((pver, ld), dtype=f64, device=T.device),
                   glambda=torch.empty(ld, dtype=f64, device=T.device),
                   gtau=torch.empty(ld, dtype=f64, device=T.device))
    if objective:
        res["P"] = torch.empty(ld, dtype=f64, device=T.device)
        res["H"] = torch.empty(ld, dtype=f64, device=T.device)
    dp = params or L.deep_defaults()
    g = vgrid.struct(n, ld)
    st = L.lib().conv_deep_adjoint(
        C.byref(g), C.byref(inp), C.byref(dp), float(dt), L.CONV_FP64, _ptr(gP), _ptr(gH), w,
        _ptr(res.get("gT")), _ptr(res.get("gq")), _ptr(res.get("glambda")),
        _ptr(res.get("gtau")), _ptr(res.get("P")), _ptr(res.get("H")), _stream(stream))
    L.check(st, "conv_deep_adjoint")
    return res


class DeepConvection(torch.autograd.Function):
    """Differentiable deep scheme: (T, q, lam, tau) -> (P, H) per column, with
    P the precipitation and H = sum_k w_k m_k cp dTdt_k.  Both directions run in
    the library: forward and backward call conv_deep_adjoint (the backward
    recomputes the forward scheme in its kernel; nothing is saved but inputs).
    lam / tau may be None (parameter defaults, no gradient)."""

    @staticmethod
    def forward(ctx, T, q, lam, tau, ps, vgrid, dt, params, w_heat):
        ctx.save_for_backward(T, q, lam, tau, ps)
        ctx.cfg = (vgrid, dt, params, w_heat)
        r = deep_adjoint(T.detach(), q.detach(), ps, vgrid, w_heat=w_heat, dt=dt,
                         lam=None if lam is None else lam.detach(),
                         tau=None if tau is None else tau.detach(), params=params,
                         gradient=False, objective=True)
        return r["P"], r["H"]

    @staticmethod
    def backward(ctx, gP, gH):
        T, q, lam, tau, ps = ctx.saved_tensors
        vgrid, dt, params, w_heat = ctx.cfg
        r = deep_adjoint(T.detach(), q.detach(), ps, vgrid, gP=gP.contiguous(),
                         gH=gH.contiguous(), w_heat=w_heat, dt=dt,
                         lam=None if lam is None else lam.detach(),
                         tau=None if tau is None else tau.detach(), params=params)
        need = ctx.needs_input_grad
        return (r["gT"] if need[0] else None, r["gq"] if need[1] else None,
                r["glambda"] if need[2] else None, r["gtau"] if need[3] else None,
                None, None, None, None, None)


def deep_precip_heating(T, q, ps, vgrid: VerticalGrid, *, lam=None, tau=None,
                        dt: float = 1800.0, params=None, w_heat=None):
    """(P, H) of the deep scheme per column, differentiable w.r.t. T, q, lam, tau."""
    return DeepConvection.apply(T, q, lam, tau, ps, vgrid, dt, params, w_heat)


def deep_shallow_adjoint(T, q, ps, vgrid: VerticalGrid, *, gPd=None, gHd=None, gPs=None,
                         gHs=None, w_heat=None, dt: float = 1800.0, lam=None, tau=None,
                         deep_params=None, shallow_params=None, n_cols=None, gradient=True,
                         objective=False, stream=None):
    """Fused-step objective and/or adjoint (FP64, conv_deep_shallow_adjoint).

    Per column: Pd, Hd, Ps, Hs (precipitation and H = sum_k w_k m_k cp dTdt_k of
    the deep and of the shallow scheme, the shallow scheme run on the
    deep-updated state), and the gradient of J = gPd Pd + gHd Hd + gPs Ps + gHs Hs
    with respect to T, q ([pver, ld]), lambda and tau ([ld]).  Returns a dict
    with gT, gq, glambda, gtau (if ``gradient``) and obj ([4, ld] rows Pd, Hd, Ps,
    Hs; if ``objective``)."""
    if not (gradient or objective):
        raise ValueError("nothing requested")
    pver, ld, n, inp = _common(T, q, ps, vgrid, n_cols, "fp64", lam, tau)
    f64 = torch.float64
    seeds = (gPd, gHd, gPs, gHs)
    for name, t in zip(("gPd", "gHd", "gPs", "gHs"), seeds):
        if t is not None:
            _require_cuda(t, name, f64, (ld,))
    w = None
    if w_heat is not None:
        wa = np.ascontiguousarray(w_heat, dtype=np.float64)
        if wa.shape != (pver,):
            raise ValueError(f"w_heat must have {pver} entries")
        w = wa.ctypes.data_as(C.POINTER(C.c_double))
    res = dict(gT=torch.empty((pver, ld), dtype=f64, device=T.device),
               gq=torch.empty((pver, ld), dtype=f64, device=T.device))
    if gradient:
        res["glambda"] = torch.empty(ld, dtype=f64, device=T.device)
        res["gtau"] = torch.empty(ld, dtype=f64, device=T.device)
    if objective:
        res["obj"] = torch.empty((4, ld), dtype=f64, device=T.device)
    dp = deep_params or L.deep_defaults()
    sp = shallow_params or L.shallow_defaults()
    g = vgrid.struct(n, ld)
    st = L.lib().conv_deep_shallow_adjoint(
        C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp), float(dt), L.CONV_FP64,
        *[_ptr(x) for x in seeds], w, _ptr(res["gT"]), _ptr(res["gq"]),
        _ptr(res.get("glambda")), _ptr(res.get("gtau")), _ptr(res.get("obj")),
        1 if gradient else 0, _stream(stream))
    L.check(st, "conv_deep_shallow_adjoint")
    if not gradient:
        del res["gT"], res["gq"]
    return res


class DeepShallowStep(torch.autograd.Function):
    """Differentiable fused step: (T, q, lam, tau) -> (Pd, Hd, Ps, Hs) per column
    (deep scheme, then shallow scheme on the deep-updated state).  Forward and
    backward both run in the library (conv_deep_shallow_adjoint); the backward
    recomputes both schemes in its kernel.  lam / tau may be None."""

    @staticmethod
    def forward(ctx, T, q, lam, tau, ps, vgrid, dt, deep_params, shallow_params, w_heat):
        ctx.save_for_backward(T, q, lam, tau, ps)
        ctx.cfg = (vgrid, dt, deep_params, shallow_params, w_heat)
        r = deep_shallow_adjoint(T.detach(), q.detach(), ps, vgrid, w_heat=w_heat, dt=dt,
                                 lam=None if lam is None else lam.detach(),
                                 tau=None if tau is None else tau.detach(),
                                 deep_params=deep_params, shallow_params=shallow_params,
                                 gradient=False, objective=True)
        o = r["obj"]
        return o[0].clone(), o[1].clone(), o[2].clone(), o[3].clone()

    @staticmethod
    def backward(ctx, gPd, gHd, gPs, gHs):
        T, q, lam, tau, ps = ctx.saved_tensors
        vgrid, dt, deep_params, shallow_params, w_heat = ctx.cfg
        r = deep_shallow_adjoint(T.detach(), q.detach(), ps, vgrid, gPd=gPd.contiguous(),
                                 gHd=gHd.contiguous(), gPs=gPs.contiguous(),
                                 gHs=gHs.contiguous(), w_heat=w_heat, dt=dt,
                                 lam=None if lam is None else lam.detach(),
                                 tau=None if tau is None else tau.detach(),
                                 deep_params=deep_params, shallow_params=shallow_params)
        need = ctx.needs_input_grad
        return (r["gT"] if need[0] else None, r["gq"] if need[1] else None,
                r["glambda"] if need[2] else None, r["gtau"] if need[3] else None,
                None, None, None, None, None, None)


def deep_shallow_step(T, q, ps, vgrid: VerticalGrid, *, lam=None, tau=None, dt: float = 1800.0,
                      deep_params=None, shallow_params=None, w_heat=None):
    """(Pd, Hd, Ps, Hs) of the fused step per column, differentiable w.r.t. T, q,
    lam, tau."""
    return DeepShallowStep.apply(T, q, lam, tau, ps, vgrid, dt, deep_params, shallow_params,
                                 w_heat)


def advance(T, q, vgrid: VerticalGrid, deep_out, shallow_out, *, dt: float, precision="fp64",
            T_relax=None, q_relax=None, tau_relax: float = 0.0, n_cols=None, stream=None):
    """In-place state advance after one fused step (conv_advance):
    T += dt*((dTdt_deep + dTdt_shallow) + (T_relax - T)/tau_relax), likewise q
    (floored at 0); tau_relax <= 0 switches the relaxation off."""
    rd = real_dtype(precision)
    pver, ld = T.shape
    _require_cuda(T, "T", rd, (pver, ld))
    _require_cuda(q, "q", rd, (pver, ld))
    if tau_relax > 0:
        _require_cuda(T_relax, "T_relax", rd, (pver, ld))
        _require_cuda(q_relax, "q_relax", rd, (pver, ld))
    n = ld if n_cols is None else int(n_cols)
    g = vgrid.struct(n, ld)
    st = L.lib().conv_advance(C.byref(g), _ptr(T), _ptr(q), _ptr(T_relax), _ptr(q_relax),
                              float(tau_relax),
                              C.byref(_out_struct(deep_out, pver, ld, precision)),
                              C.byref(_out_struct(shallow_out, pver, ld, precision)), float(dt),
                              _PREC[precision], _stream(stream))
    L.check(st, "conv_advance")


class ColumnModel:
    """Multi-step column driver: every step runs the fused deep -> shallow scheme
    on the current state and advances the state with the tendencies and a
    Newtonian relaxation (time scale tau_relax, s) towards the initial profiles,
    which stand in for the large-scale forcing of a full model.  T, q: [pver, ld]
    device tensors of the precision's type (copied); ps [ld] float64."""

    def __init__(self, T, q, ps, vgrid: VerticalGrid, *, precision="fp64", dt: float = 1800.0,
                 tau_relax: float = 86400.0, lam=None, tau=None, deep_params=None,
                 shallow_params=None, path="auto"):
        rd = real_dtype(precision)
        self.T, self.q = T.to(rd).clone(), q.to(rd).clone()
        self.T_ref, self.q_ref = self.T.clone(), self.q.clone()
        self.ps, self.vgrid, self.precision, self.dt = ps, vgrid, precision, float(dt)
        self.tau_relax, self.lam, self.tau, self.path = float(tau_relax), lam, tau, path
        self.deep_params, self.shallow_params = deep_params, shallow_params
        pver, ld = self.T.shape
        self.out_deep = new_outputs(pver, ld, precision, T.device)
        self.out_shallow = new_outputs(pver, ld, precision, T.device)
        self.ws = Workspace(T.device)
        self.steps = 0
        self._graph = None

    def _one_step(self, stream=None):
        deep_shallow(self.T, self.q, self.ps, self.vgrid, dt=self.dt, precision=self.precision,
                     lam=self.lam, tau=self.tau, deep_params=self.deep_params,
                     shallow_params=self.shallow_params, path=self.path,
                     out_deep=self.out_deep, out_shallow=self.out_shallow, workspace=self.ws,
                     stream=stream)
        advance(self.T, self.q, self.vgrid, self.out_deep, self.out_shallow, dt=self.dt,
                precision=self.precision, T_relax=self.T_ref, q_relax=self.q_ref,
                tau_relax=self.tau_relax, stream=stream)

    def step(self, n: int = 1, stream=None):
        for _ in range(n):
            self._one_step(stream)
            self.steps += 1
        return self.T, self.q

    def run_graph(self, n: int):
        """n steps replaying a CUDA graph of one step on the current stream: the
        kernels of step() in the same order, with no host work per step.  The
        first call runs one step eagerly (it loads the kernels and sizes the
        workspace) and captures the graph; later calls only replay it."""
        if n <= 0:
            return self.T, self.q
        if self._graph is None:
            self.step(1)
            n -= 1
            torch.cuda.synchronize(self.T.device)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                self._one_step()
            self._graph = graph
        for _ in range(n):
            self._graph.replay()
            self.steps += 1
        return self.T, self.q


def new_host_outputs(pver: int, ld: int, precision: str) -> dict:
    """One scheme's output tensors in page-locked host memory (for HostPipeline)."""
    rd = real_dtype(precision)
    f64, i32 = torch.float64, torch.int32
    shapes = dict(dTdt=((pver, ld), rd), dqdt=((pver, ld), rd), prec=((ld,), f64),
                  flags=((ld,), i32), kb=((ld,), i32), klcl=((ld,), i32), ktop=((ld,), i32),
                  kaux=((ld,), i32), cape=((ld,), f64), mb=((ld,), f64), cons_err=((ld,), f64))
    return {k: torch.empty(sh, dtype=dt).pin_memory() for k, (sh, dt) in shapes.items()}


def _host_ptrs(o: dict) -> L.Out:
    return L.Out(*[None if o.get(k) is None else C.c_void_p(o[k].data_ptr())
                   for k in _OUT_FIELDS])


class HostPipeline:
    """Fused deep -> shallow runs on host (page-locked) tensors, in column chunks
    whose copies in, kernels and copies out overlap on three streams
    (conv_pipeline_*).  The plan allocates its device staging once."""

    def __init__(self, vgrid: VerticalGrid, n_cols: int, ld: int, precision="mixed",
                 chunk_cols: int = 0):
        # default: four chunks (measured on the 884,736-column grid: 3.68 ms per
        # run against 3.96 with two, 4.03 with eight and 5.4 with sixteen)
        if chunk_cols <= 0:
            chunk_cols = max(65536, -(-int(n_cols) // 4))
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {list(_PREC)}")
        self.vgrid, self.n, self.ld, self.precision = vgrid, int(n_cols), int(ld), precision
        self._g = vgrid.struct(self.n, self.ld)
        h = C.c_void_p()
        L.check(L.lib().conv_pipeline_plan(C.byref(self._g), _PREC[precision], int(chunk_cols),
                                           C.byref(h)), "conv_pipeline_plan")
        self._h = h

    def run(self, T, q, ps, out_deep, out_shallow, *, dt: float = 1800.0, lam=None, tau=None,
            deep_params=None, shallow_params=None, stream=None):
        rd = real_dtype(self.precision)
        for name, t, shape, dt_ in (("T", T, (self.vgrid.pver, self.ld), rd),
                                    ("q", q, (self.vgrid.pver, self.ld), rd),
                                    ("ps", ps, (self.ld,), torch.float64)):
            if t.is_cuda or t.dtype != dt_ or tuple(t.shape) != shape or not t.is_contiguous():
                raise TypeError(f"{name} must be a contiguous host {dt_} tensor of shape {shape}")
        for name, t in (("lam", lam), ("tau", tau)):
            if t is not None and (t.is_cuda or t.dtype != torch.float64):
                raise TypeError(f"{name} must be a host float64 tensor")
        inp = L.In(C.c_void_p(T.data_ptr()), C.c_void_p(q.data_ptr()), C.c_void_p(ps.data_ptr()),
                   None if lam is None else C.c_void_p(lam.data_ptr()),
                   None if tau is None else C.c_void_p(tau.data_ptr()))
        dp = deep_params or L.deep_defaults()
        sp = shallow_params or L.shallow_defaults()
        L.check(L.lib().conv_pipeline_run(self._h, C.byref(inp), C.byref(dp), C.byref(sp),
                                          float(dt), C.byref(_host_ptrs(out_deep)),
                                          C.byref(_host_ptrs(out_shallow)), _stream(stream)),
                "conv_pipeline_run")

    def close(self):
        if getattr(self, "_h", None):
            L.lib().conv_pipeline_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
