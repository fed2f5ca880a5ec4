"""Double-float arithmetic of the FP32 path (hi + lo float pairs in place of
FP64 for the nominal trajectory, the rollout, defects and merits) checked on
the GPU against FP64: each operation within its error bound, and one RK4 step
(Eq. (1b)) of every model against the oracle's FP64 step."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2603_10711_gb300 import ucn  # noqa: E402

# a double rounds to double-float with relative error <= 2^-48; each
# operation adds a few units of 2^-48; the bound leaves a margin of ~16
EPS = 2.0 ** -44


def run(op, a, b=None, prm=None, h=0.0, nx=None):
    dev = torch.device("cuda")
    ta = torch.tensor(a, dtype=torch.float64, device=dev)
    tb = None if b is None else torch.tensor(b, dtype=torch.float64, device=dev)
    tp = None if prm is None else torch.tensor(prm, dtype=torch.float64, device=dev)
    out = torch.empty((len(a), nx) if nx else (len(a),), dtype=torch.float64, device=dev)
    ucn.ucn_df_check(op, ta, tb, tp, h, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def operands(n=20000, seed=0):
    rng = np.random.default_rng(seed)
    # magnitudes 1e-12 .. 1e12: products and quotients stay well inside the
    # float exponent range, where double-float keeps its ~48 bits
    mag = 10.0 ** rng.uniform(-12, 12, n)
    a = mag * rng.uniform(-1, 1, n)
    b = 10.0 ** rng.uniform(-12, 12, n) * rng.uniform(-1, 1, n)
    # near-cancellation: b = -a (1 + tiny)
    k = n // 4
    b[:k] = -a[:k] * (1 + rng.uniform(-1e-6, 1e-6, k))
    # exact zeros and equal magnitudes
    a[k:k + 10] = 0.0
    b[k + 10:k + 20] = a[k + 10:k + 20]
    return a, b


def test_sum_and_difference_within_the_bound():
    a, b = operands()
    for op, ref in ((ucn.UCN_DF_ADD, a + b), (ucn.UCN_DF_SUB, a - b)):
        r = run(op, a, b)
        assert np.all(np.abs(r - ref) <= EPS * (np.abs(a) + np.abs(b)) + 1e-300), op


def test_product_quotient_and_root_within_the_bound():
    a, b = operands(seed=1)
    b[b == 0.0] = 1.0
    assert np.all(np.abs(run(ucn.UCN_DF_MUL, a, b) - a * b) <= EPS * np.abs(a * b))
    q = run(ucn.UCN_DF_DIV, a, b)
    assert np.all(np.abs(q - a / b) <= EPS * np.abs(a / b))
    s = run(ucn.UCN_DF_SQRT, np.abs(a))
    assert np.all(np.abs(s - np.sqrt(np.abs(a))) <= EPS * np.sqrt(np.abs(a)))


def test_round_trip_and_exact_cases():
    a, _ = operands(seed=2)
    r = run(ucn.UCN_DF_ROUND, a)
    assert np.all(np.abs(r - a) <= 2.0 ** -47 * np.abs(a))
    # values with at most 48 significant bits survive exactly; so do sums of
    # two floats and exact squares
    x = np.array([1.0, -0.5, 3.0 + 2.0 ** -30, 1234567.0, 2.0 ** -20 * 12345.0])
    np.testing.assert_array_equal(run(ucn.UCN_DF_ROUND, x), x)
    np.testing.assert_array_equal(run(ucn.UCN_DF_ADD, x, -x), np.zeros_like(x))
    np.testing.assert_array_equal(run(ucn.UCN_DF_SQRT, np.array([4.0, 9.0, 2.0 ** 40, 0.0])),
                                  np.array([2.0, 3.0, 2.0 ** 20, 0.0]))


@pytest.mark.parametrize("kind", ["quad12", "mars7", "quat13", "mars14"])
def test_rk4_step_matches_the_fp64_oracle(kind):
    prob = {"quad12": lambda: W.quad_box(6, seed=4), "mars7": lambda: W.mars_batch(6, seed=4),
            "quat13": lambda: W.quat_study(6, seed=4), "mars14": lambda: W.mars6_batch(6, seed=4)}[kind]()
    nx, nu = oracle.model_dims(prob.model)
    for b in range(prob.batch):
        N = int(prob.N[b])
        xs = prob.xguess[prob.xoff[b]:prob.xoff[b] + N]
        us = prob.uguess[prob.uoff[b]:prob.uoff[b] + N]
        # perturb off the straight-line guess so that every term of the dynamics acts
        rng = np.random.default_rng(b)
        xs = xs + 0.05 * rng.standard_normal(xs.shape) * (np.abs(xs) + 0.1)
        us = us + 0.05 * rng.standard_normal(us.shape) * (np.abs(us) + 0.1)
        if prob.model in (ucn.UCN_MODEL_QUAT13, ucn.UCN_MODEL_MARS14):
            q0 = 6 if prob.model == ucn.UCN_MODEL_QUAT13 else 7
            xs[:, q0:q0 + 4] /= np.linalg.norm(xs[:, q0:q0 + 4], axis=1, keepdims=True)
        h = float(prob.dt[b])
        r = run(ucn.UCN_DF_RK4 + prob.model, xs, us, prob.params[b], h, nx=nx)
        ref = np.stack([oracle.rk4(prob.model, prob.params[b], h, xs[k], us[k]) for k in range(N)])
        scale = np.maximum(1.0, np.abs(ref))
        assert np.abs(r - ref).max() <= 1e-12 * scale.max(), (kind, b, np.abs(r - ref).max())


def test_rejects_an_unknown_op():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ucn.UcnError):
        ucn.ucn_df_check(9, x, x, None, 0.0, x)
    with pytest.raises(ucn.UcnError):
        ucn.ucn_df_check(ucn.UCN_DF_RK4 + 9, x, x, x, 0.1, x.view(4, 1))


def test_residual_accumulation_within_its_bound():
    # the sums of the FP32 path's ADMM residual norms: exact differences of float
    # iterates, squared and summed in double-float; a sum of t non-negative terms is
    # within (t + 8) 2^-44 of the exact sum (t = 78 here; the kernel's CTA totals add
    # at most 8 levels of a tree to each node's t terms)
    from fractions import Fraction
    rng = np.random.default_rng(5)
    t = 78
    for trial in range(20):
        a = (10.0 ** rng.uniform(-6, 2, t) * rng.uniform(-1, 1, t)).astype(np.float32).astype(np.float64)
        b = a * (1.0 + rng.uniform(-1e-3, 1e-3, t))          # near-cancelling pairs
        b[: t // 3] = (10.0 ** rng.uniform(-6, 2, t // 3)).astype(np.float32)
        b[t // 3: t // 3 + 3] = a[t // 3: t // 3 + 3]          # exact zeros
        b = b.astype(np.float32).astype(np.float64)
        exact = float(sum((Fraction(x) - Fraction(y)) ** 2 for x, y in zip(a, b)))
        dev = torch.device("cuda")
        out = torch.zeros(1, dtype=torch.float64, device=dev)
        ucn.ucn_df_check(ucn.UCN_DF_SQDIFF_SUM, torch.tensor(a, device=dev), torch.tensor(b, device=dev), None, 0.0, out)
        assert abs(float(out[0]) - exact) <= (t + 8) * EPS * exact, trial
        exact2 = float(sum(Fraction(x) ** 2 for x in a))
        ucn.ucn_df_check(ucn.UCN_DF_SQ_SUM, torch.tensor(a, device=dev), None, None, 0.0, out)
        assert abs(float(out[0]) - exact2) <= (t + 8) * EPS * exact2, trial
