"""Pins of the oracle's adjoint (the transposed Fig. 1 step run backward in
time, for the misfit 0.5*sum((T_nt - T_obs)^2)): dot-product identities of
one step against the forward step, and central finite differences of the
whole loss."""
import numpy as np
import pytest

import oracle
import synth


def _case(n, seed=4):
    g = [np.arange(k) for k in n]
    Ci = np.ascontiguousarray(synth.ci_uniform_c0(seed, *g, n))
    T0 = np.ascontiguousarray(synth.gaussian_bump(*g, n, sigma=0.2)
                              + 0.1 * synth.uniform(seed, 1, synth.global_linear_index(*g, n)))
    dd = [oracle.spacing(1.0, n[d]) for d in range(3)]
    dt = oracle.cfl_dt(*dd, 1.0, Ci.max())
    return T0, Ci, dd, dt


def test_dot_product_state_part():
    """<A x, y> = <x, A^T y> with A the (linear in T) forward step."""
    n = (9, 8, 10)
    _, Ci, dd, dt = _case(n)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((n[2], n[1], n[0]))
    y = rng.standard_normal(x.shape)
    Ax = x.copy()
    oracle.step(Ax, x, Ci, 1.3, dt, *dd)
    ATy = np.empty_like(y)
    gCi = np.zeros_like(y)
    oracle.adjoint_step(ATy, y, x, Ci, gCi, 1.3, dt, *dd)
    lhs, rhs = oracle.fsum(Ax * y), oracle.fsum(x * ATy)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), oracle.fsum(np.abs(Ax * y)))


def test_dot_product_ci_part():
    """The forward step is linear in Ci: step(Ci + h) - step(Ci) = h-part;
    <that, y> = <h, gCi(y)>."""
    n = (8, 9, 7)
    T0, Ci, dd, dt = _case(n)
    rng = np.random.default_rng(1)
    y = rng.standard_normal(T0.shape)
    h = 0.01 * rng.standard_normal(T0.shape)
    A = T0.copy()
    B = T0.copy()
    oracle.step(A, T0, Ci, 1.0, dt, *dd)
    oracle.step(B, T0, np.ascontiguousarray(Ci + h), 1.0, dt, *dd)
    gCi = np.zeros_like(T0)
    tmp = np.empty_like(T0)
    oracle.adjoint_step(tmp, y, T0, Ci, gCi, 1.0, dt, *dd)
    lhs, rhs = oracle.fsum((B - A) * y), oracle.fsum(h * gCi)
    assert abs(lhs - rhs) <= 1e-9 * oracle.fsum(np.abs(h * gCi))
    # boundary points get no Ci gradient
    inner = np.zeros(T0.shape, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert (gCi[~inner] == 0).all()


@pytest.mark.parametrize("nt", [1, 6])
def test_finite_differences(nt):
    """Central finite differences of J along random directions in Ci and T0,
    and for single entries, agree with the adjoint gradient to 1e-6."""
    n = (8, 7, 9)
    T0, Ci, dd, dt = _case(n)
    rng = np.random.default_rng(2)
    Ci_star = np.ascontiguousarray(Ci * (1 + 0.2 * rng.standard_normal(Ci.shape)))
    T_obs = oracle.forward_states(T0, Ci_star, nt, 1.0, dt, *dd)[-1]
    J, gT0, gCi = oracle.gradient(T0, Ci, T_obs, nt, 1.0, dt, *dd)
    assert J > 0

    def Jof(T0_, Ci_):
        return oracle.loss(oracle.forward_states(np.ascontiguousarray(T0_), np.ascontiguousarray(Ci_),
                                                 nt, 1.0, dt, *dd)[-1], T_obs)

    for which in ("Ci", "T0"):
        v = rng.standard_normal(T0.shape)
        base = Ci if which == "Ci" else T0
        h = 1e-6 * np.linalg.norm(base) / np.linalg.norm(v)
        if which == "Ci":
            fd = (Jof(T0, Ci + h * v) - Jof(T0, Ci - h * v)) / (2 * h)
            ad = oracle.fsum(gCi * v)
        else:
            fd = (Jof(T0 + h * v, Ci) - Jof(T0 - h * v, Ci)) / (2 * h)
            ad = oracle.fsum(gT0 * v)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (which, fd, ad)
    # single entries: one inner point, one boundary point of T0
    for (iz, iy, ix) in ((3, 3, 4), (0, 2, 3)):
        e = np.zeros_like(T0)
        e[iz, iy, ix] = 1.0
        h = 1e-5
        fd = (Jof(T0 + h * e, Ci) - Jof(T0 - h * e, Ci)) / (2 * h)
        assert abs(fd - gT0[iz, iy, ix]) <= 1e-6 * max(abs(fd), 1e-8)
    e = np.zeros_like(Ci)
    e[4, 3, 3] = 1.0
    h = 1e-6
    fd = (Jof(T0, Ci + h * e) - Jof(T0, Ci - h * e)) / (2 * h)
    assert abs(fd - gCi[4, 3, 3]) <= 1e-6 * max(abs(fd), 1e-8)


def test_bf16_rounding_definition():
    """round_to_bf16 keeps 8 significant bits with ties to even; checked
    against torch's independent BF16 conversion on FP32-representable input."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.uniform(0.3, 3.0, 4096).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to_bf16(x), ref)
    assert oracle.round_to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0      # tie -> even
    assert oracle.round_to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert np.array_equal(oracle.round_to_bf16(x), synth.bf16_bits_to_f64(synth.to_bf16_bits(x)))
