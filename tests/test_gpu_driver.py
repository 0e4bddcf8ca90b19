"""The multi-step column driver on the GPU (conv_deep_shallow_run +
conv_advance): the FP64 driver against the oracle's stepping, and the error
growth test of the paper's correctness method (Sec. V-B, after Rosinski and
Williamson): the RMS temperature difference between the mixed-precision driver
and the FP64 driver over a 2-day run (96 steps of 1800 s) must stay within the
curve of the FP64 driver with inputs perturbed in their last FP32 bit, the
induced perturbation at the mixed path's own precision."""
import numpy as np
import pytest

from paper_1711_00289_gb300 import soundings as S
from tests.gpu_util import THREADS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _model(g, precision, T=None, q=None):
    import torch

    from paper_1711_00289_gb300 import api

    T0 = torch.tensor(g.T, device="cuda") if T is None else T
    q0 = torch.tensor(g.q, device="cuda") if q is None else q
    m = api.ColumnModel(T0, q0, torch.tensor(g.ps, device="cuda"),
                        api.VerticalGrid(g.hyai, g.hybi), precision=precision, dt=g.dt)
    if T is not None:  # relax towards the unperturbed profiles
        m.T_ref = torch.tensor(g.T, device="cuda").to(m.T.dtype)
        m.q_ref = torch.tensor(g.q, device="cuda").to(m.q.dtype)
    return m


def test_fp64_driver_matches_oracle_stepping(oracle):
    import torch

    g = S.latlon_grid(24, 36)
    steps = 12
    ref = []
    oracle.column_model(g, steps, threads=THREADS,
                        record=lambda s, T, q, d, sh: ref.append((T.copy(), q.copy(), d, sh)))
    m = _model(g, "fp64")
    for s in range(steps):
        m.step()
        torch.cuda.synchronize()
        T, q = m.T.cpu().numpy(), m.q.cpu().numpy()
        Tr, qr, d, sh = ref[s]
        for o, r in ((m.out_deep, d), (m.out_shallow, sh)):
            for k in ("flags", "kb", "klcl", "ktop", "kaux"):
                assert np.array_equal(o[k].cpu().numpy(), r[k]), (s, k)
        assert np.abs(T - Tr).max() <= 1e-8, (s, np.abs(T - Tr).max())
        assert np.abs(q - qr).max() <= 1e-12, (s, np.abs(q - qr).max())


def test_error_growth_of_mixed_path_within_induced_perturbation():
    import torch

    g = S.latlon_grid(96, 144)
    steps = 96
    T0 = torch.tensor(g.T, device="cuda")
    up = torch.full_like(T0, 1e9)
    ulp64 = torch.nextafter(T0, up) - T0
    T32 = T0.float()
    ulp32 = (torch.nextafter(T32, up.float()) - T32).double()
    runs = {"fp64": _model(g, "fp64"), "lsb64": _model(g, "fp64", T=T0 + ulp64),
            "lsb32": _model(g, "fp64", T=T0 + ulp32), "mixed": _model(g, "mixed")}
    curves = {k: [] for k in ("lsb64", "lsb32", "mixed")}
    rms = lambda a, b: float(torch.sqrt(torch.mean((a.double() - b) ** 2)))
    for _ in range(steps):
        for m in runs.values():
            m.step()
        ref = runs["fp64"].T
        for k in curves:
            curves[k].append(rms(runs[k].T, ref))
    c64, c32, cm = (np.array(curves[k]) for k in ("lsb64", "lsb32", "mixed"))
    # last-bit FP64 perturbations do not grow: these column physics are not chaotic
    assert c64.max() <= 1e-12, c64.max()
    # the mixed path stays within the induced FP32 perturbation's envelope
    env = np.maximum.accumulate(c32)
    assert np.all(cm <= 2.0 * env), (cm / env).max()
    assert c32.max() < 0.5 and cm.max() < 0.5  # K: no run wanders off


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager_steps(precision):
    """ColumnModel.run_graph (one step captured into a CUDA graph, replayed)
    gives the eager steps' states bit for bit, also with the scheme variants."""
    import torch

    from paper_1711_00289_gb300 import _lib as L

    g = S.latlon_grid(48, 72)
    for dp, sp in ((None, None), ("spectrum", "evap")):
        dpar = spar = None
        if dp:
            dpar = L.deep_defaults()
            dpar.n_plumes = 3
            spar = L.shallow_defaults()
            spar.evap_k = 0.05
        runs = []
        for mode in ("eager", "graph"):
            m = _model(g, precision)
            m.deep_params, m.shallow_params = dpar, spar
            if mode == "eager":
                m.step(7)
            else:
                m.run_graph(3)
                m.run_graph(4)
            torch.cuda.synchronize()
            assert m.steps == 7
            runs.append((m.T.clone(), m.q.clone()))
        assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])
