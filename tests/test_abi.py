"""The C-ABI library loads, exports every function include/*.h declares, and
rejects invalid arguments on the host before enqueueing anything (no GPU is
touched by these tests)."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_1711_00289_gb300 import _lib as L
from paper_1711_00289_gb300 import soundings as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(conv\w*)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_declared_symbols():
    lib = L.lib()
    names = declared_functions()
    assert "conv_deep_run" in names and "conv_shallow_run" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_defaults_and_status_strings():
    dp = L.deep_defaults()
    assert dp.capelmt == 70.0 and dp.n_newton_lcl == 6 and dp.ent_zscale == 1000.0
    sp = L.shallow_defaults()
    assert sp.cin_max == 50.0 and sp.b_w == 2.0
    for s in range(6):
        assert L.status_str(s).startswith("CONV_")


def _args(pver=30, n=0, ld=0):
    # n_cols = 0: even if validation wrongly accepted an argument, nothing is
    # launched (the fake pointers below are never handed to a kernel).
    a, b = S.hybrid_coefficients(pver)
    dp = C.POINTER(C.c_double)
    g = L.Grid(pver, n, ld, 0, a.ctypes.data_as(dp), b.ctypes.data_as(dp), 1e5)
    fake = C.c_void_p(0x1000)  # never dereferenced: validation fails first
    inp = L.In(fake, fake, fake, None, None)
    out = L.Out(fake, fake, fake, fake, None, None, None, None, None, None, None)
    return g, inp, out, (a, b)


@pytest.mark.parametrize("mutate", [
    lambda g, i, o, d, s: setattr(g, "pver", 33),
    lambda g, i, o, d, s: setattr(g, "pver", 3),
    lambda g, i, o, d, s: setattr(g, "ld", -1),
    lambda g, i, o, d, s: setattr(g, "n_cols", -1),
    lambda g, i, o, d, s: setattr(i, "T", None),
    lambda g, i, o, d, s: setattr(o, "flags", None),
    lambda g, i, o, d, s: setattr(d, "tau_default", -1.0),
    lambda g, i, o, d, s: setattr(d, "n_newton_lcl", 0),
    lambda g, i, o, d, s: setattr(s, "tke", 0.0),
    lambda g, i, o, d, s: setattr(g, "p0", float("nan")),
])
def test_invalid_arguments_rejected_on_host(mutate):
    g, inp, out, keep = _args()
    dp, sp = L.deep_defaults(), L.shallow_defaults()
    mutate(g, inp, out, dp, sp)
    lib = L.lib()
    st = lib.conv_deep_shallow_run(C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp), 1800.0,
                                   L.CONV_FP64, C.byref(out), C.byref(out), None, None, 0, None)
    assert st == L.CONV_ERR_ARG


def test_unordered_levels_rejected():
    g, inp, out, (a, b) = _args()
    a2, b2 = a[::-1].copy(), b[::-1].copy()
    g.hyai = a2.ctypes.data_as(C.POINTER(C.c_double))
    g.hybi = b2.ctypes.data_as(C.POINTER(C.c_double))
    st = L.lib().conv_deep_run(C.byref(g), C.byref(inp), C.byref(L.deep_defaults()), 1800.0,
                               L.CONV_FP64, C.byref(out), None, None, 0, None)
    assert st == L.CONV_ERR_ARG


def test_bad_precision_and_dt_rejected():
    g, inp, out, keep = _args()
    lib = L.lib()
    dp = L.deep_defaults()
    assert lib.conv_deep_run(C.byref(g), C.byref(inp), C.byref(dp), 1800.0, 7, C.byref(out),
                             None, None, 0, None) == L.CONV_ERR_ARG
    assert lib.conv_deep_run(C.byref(g), C.byref(inp), C.byref(dp), -5.0, L.CONV_FP64,
                             C.byref(out), None, None, 0, None) == L.CONV_ERR_ARG
    assert lib.conv_deep_run(C.byref(g), C.byref(inp), C.byref(dp), float("inf"), L.CONV_FP64,
                             C.byref(out), None, None, 0, None) == L.CONV_ERR_ARG


def test_workspace_size_query_without_device():
    g, inp, out, keep = _args(n=1000, ld=1024)  # size query only, nothing runs
    lib = L.lib()
    plain = L.Launch(L.CONV_PATH_PLAIN, 0, 0, 0, None)
    assert lib.conv_workspace_bytes(C.byref(g), L.CONV_FP64, C.byref(plain)) == 0
    assert lib.conv_workspace_bytes(None, L.CONV_FP64, None) == 0


def test_package_has_no_cpu_fallback():
    """The product modules never import, load or run anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1711_00289_gb300")
    bad = re.compile(r"^\s*(import|from)\s+oracle\b|conv_oracle|libconv_oracle|oracle/",
                     re.M)
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            assert not bad.search(open(f).read()), f


def test_batch_plan_validates_members_before_touching_a_device():
    lib = L.lib()
    g, inp, out, keep = _args()
    m = (L.Member * 2)()
    for k in range(2):
        m[k].grid, m[k].in_, m[k].deep_out, m[k].shallow_out = g, inp, out, out
        m[k].deep, m[k].shallow, m[k].dt = L.deep_defaults(), L.shallow_defaults(), 1800.0
    m[1].deep.tau_default = -1.0
    h = C.c_void_p()
    assert lib.conv_batch_plan(m, 2, L.CONV_FP64, C.byref(h)) == L.CONV_ERR_ARG
    assert not h.value
    assert lib.conv_batch_plan(m, 0, L.CONV_FP64, C.byref(h)) == L.CONV_ERR_ARG
    assert lib.conv_batch_workspace_bytes(None) == 0
    lib.conv_batch_free(None)


def test_adjoint_arguments_checked_on_host():
    g, inp, out, keep = _args()
    dp = L.deep_defaults()
    lib = L.lib()
    fake = C.c_void_p(0x1000)
    w = (C.c_double * 30)(*([1.0] * 30))

    def call(prec=L.CONV_FP64, grads=(fake,) * 4, P=None, H=None, wh=None, dt=1800.0):
        return lib.conv_deep_adjoint(C.byref(g), C.byref(inp), C.byref(dp), dt, prec, None,
                                     None, wh, *grads, P, H, None)

    # n_cols = 0: a valid request enqueues nothing and succeeds without a device
    assert call() == L.CONV_OK
    assert call(grads=(None,) * 4, P=fake) == L.CONV_OK
    assert call(wh=w) == L.CONV_OK
    assert call(prec=L.CONV_MIXED) == L.CONV_ERR_UNSUPPORTED
    assert call(prec=7) == L.CONV_ERR_ARG
    assert call(grads=(fake, fake, None, fake)) == L.CONV_ERR_ARG
    assert call(grads=(None,) * 4) == L.CONV_ERR_ARG  # nothing requested
    assert call(dt=0.0) == L.CONV_ERR_ARG
    w[3] = float("nan")
    assert call(wh=w) == L.CONV_ERR_ARG
    dp.tau_default = 0.0
    assert call() == L.CONV_ERR_ARG


def test_step_adjoint_arguments_checked_on_host():
    g, inp, out, keep = _args()
    dp, sp = L.deep_defaults(), L.shallow_defaults()
    lib = L.lib()
    fake = C.c_void_p(0x1000)

    def call(prec=L.CONV_FP64, gT=fake, gq=fake, gl=fake, gt=fake, obj=None, grad=1):
        return lib.conv_deep_shallow_adjoint(C.byref(g), C.byref(inp), C.byref(dp),
                                             C.byref(sp), 1800.0, prec, None, None, None,
                                             None, None, gT, gq, gl, gt, obj, grad, None)

    # n_cols = 0: nothing is enqueued
    assert call() == L.CONV_OK
    assert call(gl=None, gt=None, obj=fake, grad=0) == L.CONV_OK
    assert call(prec=L.CONV_MIXED) == L.CONV_ERR_UNSUPPORTED
    assert call(gT=None) == L.CONV_ERR_ARG  # gT, gq are always needed (deep tendencies)
    assert call(gl=None) == L.CONV_ERR_ARG
    assert call(grad=0) == L.CONV_ERR_ARG  # nothing requested
    sp.tke = 0.0
    assert call() == L.CONV_ERR_ARG


def test_pipeline_plan_validated_before_touching_a_device():
    g, inp, out, keep = _args(n=10, ld=10)
    lib = L.lib()
    h = C.c_void_p()
    assert lib.conv_pipeline_plan(C.byref(g), L.CONV_MIXED, 0, C.byref(h)) == L.CONV_ERR_ARG
    assert lib.conv_pipeline_plan(C.byref(g), 7, 16, C.byref(h)) == L.CONV_ERR_ARG
    g.pver = 3
    assert lib.conv_pipeline_plan(C.byref(g), L.CONV_MIXED, 16, C.byref(h)) == L.CONV_ERR_ARG
    assert lib.conv_pipeline_run(None, C.byref(inp), C.byref(L.deep_defaults()),
                                 C.byref(L.shallow_defaults()), 1800.0, C.byref(out),
                                 C.byref(out), None) == L.CONV_ERR_ARG
    lib.conv_pipeline_free(None)


def test_tracer_transport_arguments_checked_on_host():
    """conv_tracer_transport rejects bad arguments before any launch (n_cols = 0
    throughout, so nothing would run even if a check were missing)."""
    g, _, out, keep = _args()
    lib = L.lib()
    fake = C.c_void_p(0x1000)
    flux = L.Out(fake, fake, fake, fake, fake, None, fake, fake, None, None, None, fake, fake, fake)

    def call(d, s, ntr=1, tr=fake, td=fake, ts=fake, dt=1800.0, prec=L.CONV_FP64, ps=fake):
        return lib.conv_tracer_transport(C.byref(g), ps, None if d is None else C.byref(d),
                                         None if s is None else C.byref(s), dt, ntr, tr, td, ts,
                                         prec, None)

    assert call(flux, flux) == L.CONV_OK  # valid (nothing to do for 0 columns)
    assert call(None, None) == L.CONV_ERR_ARG
    assert call(flux, flux, ntr=-1) == L.CONV_ERR_ARG
    assert call(flux, flux, tr=None) == L.CONV_ERR_ARG
    assert call(flux, flux, ps=None) == L.CONV_ERR_ARG
    assert call(flux, None, td=None) == L.CONV_ERR_ARG
    assert call(None, flux, ts=None) == L.CONV_ERR_ARG
    assert call(flux, flux, dt=0.0) == L.CONV_ERR_ARG
    assert call(flux, flux, prec=7) == L.CONV_ERR_ARG
    assert call(None, out) == L.CONV_ERR_ARG  # no mass-flux profiles in this output set
    no_kaux = L.Out(fake, fake, fake, fake, fake, None, fake, None, None, None, None, fake, fake,
                    fake)
    assert call(no_kaux, None) == L.CONV_ERR_ARG  # deep downdraft without its top layer
    assert call(None, no_kaux) == L.CONV_OK  # the shallow scheme has no downdraft


def test_batch_rejects_mass_flux_outputs():
    g, inp, out, keep = _args(n=0)
    fake = C.c_void_p(0x1000)
    mb = L.Member()
    mb.grid, mb.in_ = g, inp
    mb.deep_out = L.Out(fake, fake, fake, fake, None, None, None, None, None, None, None, fake)
    mb.shallow_out = out
    mb.deep, mb.shallow = L.deep_defaults(), L.shallow_defaults()
    mb.dt = 1800.0
    h = C.c_void_p()
    st = L.lib().conv_batch_plan(C.byref(mb), 1, L.CONV_FP64, C.byref(h))
    assert st == L.CONV_ERR_UNSUPPORTED


def test_evaporation_variant_arguments():
    """A negative or non-finite evaporation coefficient is rejected; the variant
    is refused by the batched runs and by the fused-step adjoint (no adjoint of
    it), all before any device work."""
    g, inp, out, keep = _args()
    lib = L.lib()
    dp, sp = L.deep_defaults(), L.shallow_defaults()
    assert sp.evap_k == 0.0
    for bad in (-1.0, float("nan"), float("inf")):
        sp.evap_k = bad
        st = lib.conv_deep_shallow_run(C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp),
                                       1800.0, L.CONV_FP64, C.byref(out), C.byref(out), None,
                                       None, 0, None)
        assert st == L.CONV_ERR_ARG
    sp.evap_k = 0.05
    mb = L.Member()
    mb.grid, mb.in_, mb.deep_out, mb.shallow_out = g, inp, out, out
    mb.deep, mb.shallow, mb.dt = dp, sp, 1800.0
    h = C.c_void_p()
    assert lib.conv_batch_plan(C.byref(mb), 1, L.CONV_FP64, C.byref(h)) == L.CONV_ERR_UNSUPPORTED
    fake = C.c_void_p(0x1000)
    st = lib.conv_deep_shallow_adjoint(C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp),
                                       1800.0, L.CONV_FP64, None, None, None, None, None, fake,
                                       fake, fake, fake, None, 1, None)
    assert st == L.CONV_ERR_UNSUPPORTED


def test_plume_spectrum_arguments():
    """n_plumes outside 1..CONV_MAX_PLUMES or a spread below 1 is rejected; the
    variant is refused with mass-flux profile outputs, by batched runs and by
    both adjoints, all before any device work."""
    g, inp, out, keep = _args()
    lib = L.lib()
    dp, sp = L.deep_defaults(), L.shallow_defaults()
    assert dp.n_plumes == 1 and dp.plume_spread == 4.0

    def run(d, o=out):
        return lib.conv_deep_shallow_run(C.byref(g), C.byref(inp), C.byref(d), C.byref(sp),
                                         1800.0, L.CONV_FP64, C.byref(o), C.byref(o), None,
                                         None, 0, None)

    for n, spread in ((0, 4.0), (9, 4.0), (3, 0.5), (3, float("nan"))):
        dp.n_plumes, dp.plume_spread = n, spread
        assert run(dp) == L.CONV_ERR_ARG
    dp.n_plumes, dp.plume_spread = 3, 4.0
    fake = C.c_void_p(0x1000)
    flux = L.Out(fake, fake, fake, fake, None, None, None, None, None, None, None, fake)
    assert run(dp, flux) == L.CONV_ERR_UNSUPPORTED
    mb = L.Member()
    mb.grid, mb.in_, mb.deep_out, mb.shallow_out = g, inp, out, out
    mb.deep, mb.shallow, mb.dt = dp, sp, 1800.0
    h = C.c_void_p()
    assert lib.conv_batch_plan(C.byref(mb), 1, L.CONV_FP64, C.byref(h)) == L.CONV_ERR_UNSUPPORTED
    st = lib.conv_deep_adjoint(C.byref(g), C.byref(inp), C.byref(dp), 1800.0, L.CONV_FP64,
                               None, None, None, fake, fake, fake, fake, None, None, None)
    assert st == L.CONV_ERR_UNSUPPORTED
    st = lib.conv_deep_shallow_adjoint(C.byref(g), C.byref(inp), C.byref(dp), C.byref(sp),
                                       1800.0, L.CONV_FP64, None, None, None, None, None, fake,
                                       fake, fake, fake, None, 1, None)
    assert st == L.CONV_ERR_UNSUPPORTED


@pytest.mark.parametrize("which,k,val", [("a", -1, float("nan")), ("b", -1, float("inf")),
                                         ("a", 0, float("nan")), ("b", 12, float("nan"))])
def test_non_finite_level_coefficients_rejected(which, k, val):
    """Every one of the pver + 1 interface coefficients must be finite, the
    surface interface included (a NaN there compares false in the ordering
    check, so finiteness is checked on its own)."""
    g, inp, out, (a, b) = _args()
    arr = (a if which == "a" else b).copy()
    arr[k] = val
    dp = C.POINTER(C.c_double)
    if which == "a":
        g.hyai = arr.ctypes.data_as(dp)
    else:
        g.hybi = arr.ctypes.data_as(dp)
    st = L.lib().conv_deep_run(C.byref(g), C.byref(inp), C.byref(L.deep_defaults()), 1800.0,
                               L.CONV_FP64, C.byref(out), None, None, 0, None)
    assert st == L.CONV_ERR_ARG


def test_pipeline_checks_everything_before_its_first_copy():
    """A pipeline run refuses bad parameter blocks, dt and missing required host
    outputs before it touches its plan or enqueues a copy, so an error return
    never leaves copies of the caller's buffers in flight (the plan handle below
    is never dereferenced); a plan refuses a level table a run would refuse."""
    g, inp, out, (a, b) = _args(n=10, ld=10)
    lib = L.lib()
    plan = C.c_void_p(0x1000)
    fake = C.c_void_p(0x1000)

    def run(dp=None, sp=None, dt=1800.0, od=out, os_=out):
        return lib.conv_pipeline_run(plan, C.byref(inp), C.byref(dp or L.deep_defaults()),
                                     C.byref(sp or L.shallow_defaults()), dt, C.byref(od),
                                     C.byref(os_), None)

    bad_d = L.deep_defaults()
    bad_d.tau_default = -1.0
    bad_s = L.shallow_defaults()
    bad_s.tke = 0.0
    no_prec = L.Out(fake, fake, None, fake, None, None, None, None, None, None, None)
    assert run(dp=bad_d) == L.CONV_ERR_ARG
    assert run(sp=bad_s) == L.CONV_ERR_ARG
    assert run(dt=0.0) == L.CONV_ERR_ARG
    assert run(dt=float("nan")) == L.CONV_ERR_ARG
    assert run(od=no_prec) == L.CONV_ERR_ARG
    assert run(os_=no_prec) == L.CONV_ERR_ARG
    a2 = a.copy()
    a2[-1] = float("nan")
    g.hyai = a2.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    assert lib.conv_pipeline_plan(C.byref(g), L.CONV_MIXED, 16, C.byref(h)) == L.CONV_ERR_ARG
    a3, b3 = a[::-1].copy(), b[::-1].copy()  # surface first: interfaces out of order
    g.hyai = a3.ctypes.data_as(C.POINTER(C.c_double))
    g.hybi = b3.ctypes.data_as(C.POINTER(C.c_double))
    assert lib.conv_pipeline_plan(C.byref(g), L.CONV_MIXED, 16, C.byref(h)) == L.CONV_ERR_ARG
    assert not h.value
