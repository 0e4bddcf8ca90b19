"""The mixed path's FP32 quotient (conv_bench_f32_quotient: the division of every
FP32 step of the schemes, PTX div.full.f32 in the default build) against IEEE
division computed on the host by numpy: within 2 ulp on random operands of
magnitudes 2^-20 .. 2^20 and on the operand ranges of the saturation formulas,
and IEEE's results for division by zero and infinity."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _quotient(a, b):
    import torch

    from paper_1711_00289_gb300 import _lib as L

    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    dq = torch.empty_like(da)
    L.f32_quotient(da.data_ptr(), db.data_ptr(), dq.data_ptr(), a.size)
    torch.cuda.synchronize()
    return dq.cpu().numpy()


def _ordered(x):
    i = x.view(np.int32).astype(np.int64)
    return np.where(i < 0, -(i & 0x7FFFFFFF), i)


def ulp_distance(x, y):
    return np.abs(_ordered(x) - _ordered(y))


def _random_operands(seed, n):
    rng = np.random.default_rng(seed)
    sign = rng.choice(np.array([-1.0, 1.0]), size=n)
    return (sign * np.exp2(rng.uniform(-20.0, 20.0, size=n))).astype(np.float32)


def test_random_operands_within_two_ulp():
    n = 1 << 22
    a, b = _random_operands(1, n), _random_operands(2, n)
    q = _quotient(a, b)
    ref = a / b
    assert ref.dtype == np.float32
    d = ulp_distance(q, ref)
    assert d.max() <= 2, (int(d.max()), a[d.argmax()], b[d.argmax()])


def test_saturation_formula_operands():
    """The quotients of the saturation formulas: 1/(T - 29.65), 17.67 (T -
    273.15)/(T - 29.65), eps es / D with D in 1..1100 hPa."""
    rng = np.random.default_rng(3)
    T = rng.uniform(150.0, 350.0, size=1 << 20).astype(np.float32)
    es = rng.uniform(1e-3, 8e3, size=T.size).astype(np.float32)
    D = rng.uniform(1e2, 1.1e5, size=T.size).astype(np.float32)
    cases = [(np.ones_like(T), T - np.float32(29.65)),
             (np.float32(17.67) * (T - np.float32(273.15)), T - np.float32(29.65)),
             (np.float32(0.622) * es, D)]
    for a, b in cases:
        d = ulp_distance(_quotient(a, b), a / b)
        assert d.max() <= 2, int(d.max())


def test_zero_and_infinite_operands():
    inf = np.float32(np.inf)
    a = np.array([1.0, -1.0, 0.0, 0.0, 5.0, -5.0, 3.0], dtype=np.float32)
    b = np.array([0.0, 0.0, 5.0, -5.0, inf, inf, 3.0], dtype=np.float32)
    q = _quotient(a, b)
    assert q[0] == inf and q[1] == -inf
    assert q[2] == 0 and q[3] == 0 and q[4] == 0 and q[5] == 0
    assert q[6] == 1.0
    assert np.isnan(_quotient(np.zeros(1, np.float32), np.zeros(1, np.float32))[0])


def test_empty_and_bad_arguments():
    from paper_1711_00289_gb300 import _lib as L

    L.f32_quotient(0, 0, 0, 0)  # n = 0: nothing to do, null pointers allowed
    with pytest.raises(L.ConvError):
        L.f32_quotient(0, 0, 0, 5)
    with pytest.raises(L.ConvError):
        L.f32_quotient(0, 0, 0, -1)
