"""Pins of the FP64 oracle against facts it does not compute itself (CPU only).

Each check ties an oracle function to the mathematics: closed-form point counts, circular
convolution by numpy's FFT, plane-wave eigenvalues, exactness of central differences on
polynomials, transpose identities, numpy/torch rounding, and finite differences of the wave
misfit.  A dropped term, a flipped sign or index, or a transposed operand in the oracle fails
at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2609_06694_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
SHAPES = ["star", "box", "diamond"]


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# --------------------------------------------------------------------------------------------
# offset sets
# --------------------------------------------------------------------------------------------

def _golden_counts():
    rows = []
    with open(os.path.join(HERE, "golden", "offset_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                nd, shape, r, n = line.split()
                rows.append((int(nd), shape, int(r), int(n)))
    return rows


@pytest.mark.parametrize("ndim,shape,r,n", _golden_counts())
def test_offset_counts_match_golden(ndim, shape, r, n):
    assert len(oracle.offsets(ndim, shape, r)) == n


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_offset_sets_definition(ndim, shape, r):
    offs = oracle.offsets(ndim, shape, r)
    # membership by the norms of Sec. 2.1 (star: on an axis; box: inf-norm; diamond: 1-norm)
    want = []
    for d in itertools.product(range(-r, r + 1), repeat=ndim):
        nz = sum(1 for x in d if x)
        if shape == "star" and nz > 1:
            continue
        if shape == "diamond" and sum(abs(x) for x in d) > r:
            continue
        want.append(d)
    got = [tuple(int(x) for x in o) for o in offs]
    assert got == want  # itertools.product is lexicographic: the canonical order
    assert max(max(abs(x) for x in o) for o in got) == r  # order r = max inf-norm
    assert set(got) == {tuple(-x for x in o) for o in got}  # closed under negation


# --------------------------------------------------------------------------------------------
# constant-coefficient sweep
# --------------------------------------------------------------------------------------------

def fft_periodic_sweep(x, offs, c):
    """out[p] = sum_o c_o x[p+o] (circular) as a convolution with a kernel at -o, via FFT."""
    k = np.zeros(x.shape)
    for o, w in zip(offs, c):
        idx = tuple((-int(d)) % n for d, n in zip(o, x.shape))
        k[idx] += w
    return np.real(np.fft.ifftn(np.fft.fftn(x) * np.fft.fftn(k)))


def fft_periodic_adjoint(y, offs, c):
    """(A^T y)[q] = sum_o c_o y[q-o] (circular): kernel at +o."""
    k = np.zeros(y.shape)
    for o, w in zip(offs, c):
        idx = tuple(int(d) % n for d, n in zip(o, y.shape))
        k[idx] += w
    return np.real(np.fft.ifftn(np.fft.fftn(y) * np.fft.fftn(k)))


GRIDS = {2: [(13, 11), (3, 5), (16, 16)], 3: [(7, 6, 9), (3, 2, 5), (8, 8, 8)]}


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2, 4])
def test_periodic_sweep_is_circular_convolution(ndim, shape, r):
    offs = oracle.offsets(ndim, shape, r)
    for g, dims in enumerate(GRIDS[ndim]):
        c = inputs.uniform(700 + 10 * r + g, (len(offs),))
        x = inputs.uniform(800 + 10 * r + g, dims)
        got = oracle.sweep_const(x, offs, c, "periodic")
        assert relerr(got, fft_periodic_sweep(x, offs, c)) < 1e-12
        got_t = oracle.sweep_const_adjoint(x, offs, c, "periodic")
        assert relerr(got_t, fft_periodic_adjoint(x, offs, c)) < 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 3])
def test_dirichlet_sweep_is_zero_padded_convolution(ndim, shape, r):
    """Ghost zeros: the sweep equals a circular convolution of the input padded by r zeros."""
    offs = oracle.offsets(ndim, shape, r)
    dims = GRIDS[ndim][0]
    c = inputs.uniform(900 + r, (len(offs),))
    x = inputs.uniform(901 + r, dims)
    pad = np.pad(x, r)
    full = fft_periodic_sweep(pad, offs, c)
    crop = full[tuple(slice(r, r + n) for n in dims)]
    assert relerr(oracle.sweep_const(x, offs, c, "dirichlet"), crop) < 1e-12
    full_t = fft_periodic_adjoint(pad, offs, c)
    crop_t = full_t[tuple(slice(r, r + n) for n in dims)]
    assert relerr(oracle.sweep_const_adjoint(x, offs, c, "dirichlet"), crop_t) < 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2, 3, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_point_evaluation_is_the_sweep_at_every_cell(ndim, shape, r, bc):
    """The point evaluator (the reference of the full-size spot checks) against the FFT
    convolution at every cell of small grids -- corners, edges, faces and, for periodic grids
    smaller than the stencil, cells whose reads wrap several times -- in a shuffled order with
    repeats, and bit for bit against the whole-grid sweep."""
    offs = oracle.offsets(ndim, shape, r)
    for g, dims in enumerate(GRIDS[ndim]):
        c = inputs.uniform(950 + 10 * r + g, (len(offs),))
        x = inputs.uniform(960 + 10 * r + g, dims)
        if bc == "periodic":
            want = fft_periodic_sweep(x, offs, c)
        else:
            pad = np.pad(x, r)
            want = fft_periodic_sweep(pad, offs, c)[tuple(slice(r, r + n) for n in dims)]
        n = int(np.prod(dims))
        sel = np.random.default_rng(g).permutation(np.concatenate([np.arange(n), [0, n - 1]]))
        got = oracle.sweep_const_points(x, offs, c, bc, sel)
        assert relerr(got, want.ravel()[sel]) < 1e-12
        assert np.array_equal(got, oracle.sweep_const(x, offs, c, bc).ravel()[sel])


@pytest.mark.parametrize("shape,r", [("star", 2), ("box", 1)])
def test_dependency_slab_reproduces_the_periodic_sweep(shape, r):
    """The slab the full-size GPU checks compare whole planes on: a Dirichlet run of the
    periodically padded slab equals the periodic run on the middle plane, including grids
    smaller than the slab (several wraps)."""
    import sys
    sys.path.insert(0, HERE)
    from helpers import periodic_slab
    offs = oracle.offsets(3, shape, r)
    c = inputs.normalised_abs_weights(980, len(offs))
    for dims, steps in (((12, 9, 10), 3), ((5, 4, 6), 2)):
        x = inputs.uniform(981, dims)
        full = oracle.run(x, "const", "periodic", steps, offs=offs, coeffs=c)
        h = steps * r
        for z0 in (0, dims[0] // 2, dims[0] - 1):
            part = oracle.run(periodic_slab(x, z0, h), "const", "dirichlet", steps, offs=offs,
                              coeffs=c)[h, h:-h, h:-h]
            assert relerr(part, full[z0]) < 1e-13


# --------------------------------------------------------------------------------------------
# reaction-diffusion (stencil fused with pointwise physics)
# --------------------------------------------------------------------------------------------

def test_reaction_without_diffusion_is_a_scalar_ode_per_cell():
    """Zero weights: every cell follows explicit Euler for u' = c1 u + c3 u^3 on its own,
    computed here cell by cell in plain Python with the same FP64 operations."""
    offs = oracle.offsets(3, "star", 2)
    x = inputs.uniform(990, (4, 5, 6))
    dt, c1, c3, steps = 0.05, 3.0, -2.5, 7
    got = oracle.reaction(x, offs, np.zeros(len(offs)), "periodic", steps, dt, c1, c3)
    for idx in ((0, 0, 0), (3, 4, 5), (2, 1, 3)):
        u = float(x[idx])
        for _ in range(steps):
            u = u + dt * (0.0 + c1 * u + c3 * u * u * u)
        assert got[idx] == u


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_reaction_linear_part_is_the_sweep_of_identity_plus_dt_a(bc):
    """c1 = c3 = 0: one step is the sweep with weights dt * c and 1 added at the centre."""
    offs = oracle.offsets(3, "box", 1)
    c = inputs.uniform(991, (len(offs),))
    x = inputs.uniform(992, (6, 7, 8))
    dt = 0.3
    w = dt * c
    w[[i for i, o in enumerate(offs) if not np.any(o)][0]] += 1.0
    want = oracle.run(x, "const", bc, 2, offs=offs, coeffs=w)
    got = oracle.reaction(x, offs, c, bc, 2, dt, 0.0, 0.0)
    assert relerr(got, want) < 1e-13


def test_reaction_constant_field_closed_form():
    """A constant field on a periodic grid stays constant: u <- u + dt (u sum(c) + c1 u +
    c3 u^3), iterated as a scalar recurrence; the linear reaction term c1 shifts it as a
    weight on the centre would."""
    offs = oracle.offsets(2, "star", 1)
    c = np.array([0.5, 1.0, -4.0, 1.0, 0.25])
    dt, c1, c3 = 0.01, 2.0, -1.0
    x = np.full((9, 11), 0.3)
    got = oracle.reaction(x, offs, c, "periodic", 5, dt, c1, c3)
    u = 0.3
    for _ in range(5):
        u = u + dt * (u * np.sum(c) + c1 * u + c3 * u ** 3)
    assert relerr(got, np.full_like(x, u)) < 1e-14


def test_threaded_build_gives_the_same_bits():
    """The OpenMP build of the oracle splits cell loops over threads only: every function used
    by the parity tests returns identical bits to the single-threaded build."""
    dims = (9, 14, 33)
    offs = oracle.offsets(3, "box", 2)
    c = inputs.uniform(970, (len(offs),))
    x = inputs.uniform(971, dims)
    k = 1.0 + inputs.uniform(972, dims) ** 2
    sel = np.arange(0, x.size, 7)

    def everything():
        return [oracle.sweep_const(x, offs, c, "periodic"),
                oracle.sweep_const_adjoint(x, offs, c, "dirichlet"),
                oracle.sweep_const_points(x, offs, c, "periodic", sel),
                oracle.divkgrad(x, k, "dirichlet"),
                oracle.run(x, "const", "dirichlet", 3, offs=offs, coeffs=c, round_fmt="bf16"),
                oracle.run(x, "divkgrad", "periodic", 2, coeffs=k, round_fmt="f16")]

    assert oracle.threads() == 1
    one = everything()
    try:
        assert oracle.use_threads(4) >= 1
        many = everything()
    finally:
        oracle.use_threads(1)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", SHAPES)
def test_single_impulse_gives_flipped_weights_clipped(shape):
    offs = oracle.offsets(3, shape, 2)
    c = np.arange(1, len(offs) + 1, dtype=np.float64)
    dims = (6, 5, 7)
    q = (1, 3, 5)  # near several faces, so some taps fall outside
    x = np.zeros(dims)
    x[q] = 1.0
    out = oracle.sweep_const(x, offs, c, "dirichlet")
    want = np.zeros(dims)
    for o, w in zip(offs, c):
        p = tuple(qq - int(d) for qq, d in zip(q, o))
        if all(0 <= pp < n for pp, n in zip(p, dims)):
            want[p] = w
    assert np.array_equal(out, want)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_constant_field_gives_weight_sum(ndim, shape):
    offs = oracle.offsets(ndim, shape, 2)
    c = inputs.uniform(31, (len(offs),))
    x = np.full(GRIDS[ndim][0], 0.75)
    out = oracle.sweep_const(x, offs, c, "periodic")
    assert np.allclose(out, 0.75 * c.sum(), rtol=0, atol=1e-14)


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_central_laplacian_exact_on_polynomials(r):
    """Order-2r central second differences are exact for polynomials of degree <= 2r+1."""
    offs = oracle.offsets(3, "star", r)
    c = inputs.laplacian_coeffs(offs, r)
    n = 2 * r + 7
    z, y, x = np.meshgrid(*[np.arange(n, dtype=np.float64) - n // 2] * 3, indexing="ij")
    deg = 2 * r + 1
    u = x ** deg + 0.5 * y ** (deg - 1) * z + z ** 2 - 3.0 * x * y * z
    lap = (deg * (deg - 1) * x ** (deg - 2) + 0.5 * (deg - 1) * (deg - 2) * y ** (deg - 3) * z
           + 2.0)
    out = oracle.sweep_const(u, offs, c, "dirichlet")
    interior = tuple(slice(r, n - r) for _ in range(3))
    assert relerr(out[interior], lap[interior]) < 1e-12


def test_central_laplacian_r4_on_x8():
    """The radius-4 weights are exact up to degree 9: the Laplacian of x^8 is 56 x^6."""
    offs = oracle.offsets(3, "star", 4)
    c = inputs.laplacian_coeffs(offs, 4)
    n = 13
    x = np.broadcast_to(np.arange(n, dtype=np.float64) - 6, (n, n, n))
    out = oracle.sweep_const(x ** 8, offs, c, "periodic")
    inner = (slice(4, 9),) * 3
    assert relerr(out[inner], (56.0 * x ** 6)[inner]) < 1e-12
    assert abs(c.sum()) < 1e-14  # Laplacian weights sum to zero


@pytest.mark.parametrize("ndim", [2, 3])
def test_mirror_symmetric_input_gives_mirror_symmetric_output(ndim):
    offs = oracle.offsets(ndim, "box", 2)
    # weights symmetric under reversal of the last axis
    base = inputs.uniform(41, (len(offs),))
    index = {tuple(int(v) for v in o): i for i, o in enumerate(offs)}
    c = np.array([base[i] + base[index[tuple(o[:-1]) + (-o[-1],)]]
                  for i, o in enumerate(map(tuple, offs))])
    dims = GRIDS[ndim][0]
    x = inputs.uniform(42, dims)
    x = x + np.flip(x, axis=-1)
    out = oracle.sweep_const(x, offs, c, "dirichlet")
    assert relerr(out, np.flip(out, axis=-1)) < 1e-13
    # periodic: mirror about index 0 (i -> -i mod n) is a flip followed by a roll of one
    xp = x + np.roll(np.flip(x, axis=-1), 1, axis=-1)
    outp = oracle.sweep_const(xp, offs, c, "periodic")
    assert relerr(outp, np.roll(np.flip(outp, axis=-1), 1, axis=-1)) < 1e-13


# --------------------------------------------------------------------------------------------
# several steps
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("steps", [1, 3, 8])
def test_plane_wave_eigenvalue_power(shape, steps):
    """Periodic: A e^{i theta.x} = lambda(theta) e^{i theta.x}, lambda = sum_o c_o e^{i theta.o}."""
    dims = (8, 6, 10)
    offs = oracle.offsets(3, shape, 1)
    # a dominant centre keeps |lambda| >= 0.4 so lambda^8 stays far above rounding
    c = 0.3 * inputs.normalised_abs_weights(51, len(offs))
    c[[i for i, o in enumerate(offs) if not np.any(o)][0]] += 0.7
    kvec = (1, 2, 3)
    theta = [2 * np.pi * k / n for k, n in zip(kvec, dims)]
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    phase = sum(t * g for t, g in zip(theta, grids))
    lam = sum(w * np.exp(1j * sum(t * int(d) for t, d in zip(theta, o))) for o, w in zip(offs, c))
    x = np.cos(phase)
    want = np.real(lam ** steps * np.exp(1j * phase))
    # sum |c| = 1 and |x| <= 1, so each step adds at most ~npts * 2^-53 of absolute error
    tol = 1e-13 * steps
    got = oracle.run(x, "const", "periodic", steps, offs=offs, coeffs=c)
    assert np.max(np.abs(got - want)) < tol
    got_t = oracle.run(x, "const", "periodic", steps, offs=offs, coeffs=c, adjoint=True)
    want_t = np.real(np.conj(lam) ** steps * np.exp(1j * phase))
    assert np.max(np.abs(got_t - want_t)) < tol
    assert np.max(np.abs(want)) > 1e3 * tol  # the check is not vacuous


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_run_equals_repeated_fft_sweeps(bc):
    dims = (9, 7)
    offs = oracle.offsets(2, "box", 2)
    c = inputs.normalised_abs_weights(61, len(offs))
    x = inputs.uniform(62, dims)
    want = x.copy()
    for _ in range(5):
        if bc == "periodic":
            want = fft_periodic_sweep(want, offs, c)
        else:
            want = fft_periodic_sweep(np.pad(want, 2), offs, c)[2:-2, 2:-2]
    assert relerr(oracle.run(x, "const", bc, 5, offs=offs, coeffs=c), want) < 1e-12


# --------------------------------------------------------------------------------------------
# variable coefficients and div(k grad u)
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("shape", SHAPES)
def test_var_sweep_coefficient_read_at_output_point(bc, shape):
    """w_o[p] = c_o m[p]  =>  A x = m (.) (C x): the coefficient belongs to the output cell."""
    dims = (5, 6, 7)
    offs = oracle.offsets(3, shape, 1)
    c = inputs.uniform(71, (len(offs),))
    m = inputs.uniform(72, dims, 0.5, 2.0)
    x = inputs.uniform(73, dims)
    w = c[:, None, None, None] * m[None]
    assert relerr(oracle.sweep_var(x, offs, w, bc), m * oracle.sweep_const(x, offs, c, bc)) < 1e-13
    # the adjoint gathers the coefficient at the source cell: A^T y = C^T (m (.) y)
    assert relerr(oracle.sweep_var_adjoint(x, offs, w, bc),
                  oracle.sweep_const_adjoint(m * x, offs, c, bc)) < 1e-13


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_dot_test_adjoint(bc, ndim, shape):
    """<A x, y> = <x, A^T y> to 1e-12 for constant and variable coefficients."""
    dims = GRIDS[ndim][0]
    offs = oracle.offsets(ndim, shape, 2)
    c = inputs.uniform(81, (len(offs),))
    w = inputs.uniform(82, (len(offs),) + dims)
    x = inputs.uniform(83, dims)
    y = inputs.uniform(84, dims)
    for fwd, adj, coef in ((oracle.sweep_const, oracle.sweep_const_adjoint, c),
                           (oracle.sweep_var, oracle.sweep_var_adjoint, w)):
        lhs = float(np.sum(fwd(x, offs, coef, bc) * y))
        rhs = float(np.sum(x * adj(y, offs, coef, bc)))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    # multi-step: (A^T)^T
    ax = oracle.run(x, "var", bc, 3, offs=offs, coeffs=w)
    aty = oracle.run(y, "var", bc, 3, offs=offs, coeffs=w, adjoint=True)
    lhs, rhs = float(np.sum(ax * y)), float(np.sum(x * aty))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_divkgrad_with_unit_k_is_seven_point_laplacian(bc):
    dims = (6, 7, 8)
    u = inputs.uniform(91, dims)
    offs = oracle.offsets(3, "star", 1)
    c = inputs.laplacian_coeffs(offs, 1)  # [1 ... -6 ... 1]
    assert sorted(c.tolist()) == [-6.0, 1, 1, 1, 1, 1, 1]
    out = oracle.divkgrad(u, np.ones(dims), bc)
    if bc == "periodic":
        want = fft_periodic_sweep(u, offs, c)
    else:
        want = fft_periodic_sweep(np.pad(u, 1), offs, c)[1:-1, 1:-1, 1:-1]
    assert relerr(out, want) < 1e-13


def test_divkgrad_linear_u_gives_central_difference_of_k():
    """u = x  =>  interior out = (k[x+1] - k[x-1]) / 2 (the face mean of k)."""
    dims = (5, 4, 9)
    k = inputs.lognormal_k(101, dims, smooth=1)
    u = np.broadcast_to(np.arange(dims[2], dtype=np.float64), dims).copy()
    out = oracle.divkgrad(u, k, "dirichlet")
    want = 0.5 * (k[:, :, 2:] - k[:, :, :-2])
    # y and z faces see a constant u, so only interior-y/z cells are free of ghost terms
    assert relerr(out[1:-1, 1:-1, 1:-1], want[1:-1, 1:-1, :]) < 1e-13


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("ndim", [2, 3])
def test_divkgrad_symmetric_seminegative_conservative(bc, ndim):
    dims = GRIDS[ndim][0]
    k = inputs.lognormal_k(111, dims)
    u = inputs.uniform(112, dims)
    v = inputs.uniform(113, dims)
    au = oracle.divkgrad(u, k, bc)
    av = oracle.divkgrad(v, k, bc)
    assert abs(np.sum(au * v) - np.sum(u * av)) < 1e-12 * np.sum(np.abs(au * v))
    assert np.sum(au * u) <= 0.0
    if bc == "periodic":
        assert abs(np.sum(au)) < 1e-12 * np.sum(np.abs(au))  # fluxes telescope
        assert np.max(np.abs(oracle.divkgrad(np.full(dims, 2.5), k, bc))) < 1e-13
    # the per-offset coefficient form is the same operator
    w = oracle.divkgrad_weights(k, bc)
    offs = oracle.offsets(ndim, "star", 1)
    assert relerr(oracle.sweep_var(u, offs, w, bc), au) < 1e-13
    # and its transpose (via the general adjoint) equals the operator itself
    assert relerr(oracle.run(u, "divkgrad", bc, 1, coeffs=k, adjoint=True), au) < 1e-13


# --------------------------------------------------------------------------------------------
# rounding to storage formats
# --------------------------------------------------------------------------------------------

def _rounding_probe_values():
    rng = np.random.default_rng(7)
    vals = [rng.standard_normal(2000) * 10.0 ** rng.integers(-9, 6, 2000),
            np.array([0.0, -0.0, 1.0, -1.0, 65504.0, 65519.9, 65520.0, 1e6, -1e6, 6e-8, 3e-8,
                      2.9e-8, 1e-10])]
    # exact ties for binary16: 1 + (2k+1) 2^-11
    vals.append(1.0 + (2 * np.arange(50) + 1) * 2.0 ** -11)
    vals.append(-(2.0 ** -14) * (1.0 + (2 * np.arange(50) + 1) * 2.0 ** -11))
    return np.concatenate(vals)


def test_round_f16_matches_numpy():
    x = _rounding_probe_values()
    got = oracle.round_to(x, "f16")
    with np.errstate(over="ignore"):
        want = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, want)


def test_round_f32_matches_numpy():
    x = _rounding_probe_values()
    x = np.concatenate([x, 1.0 + (2 * np.arange(50) + 1) * 2.0 ** -24])
    assert np.array_equal(oracle.round_to(x, "f32"), x.astype(np.float32).astype(np.float64))


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    x = _rounding_probe_values().astype(np.float32).astype(np.float64)  # exact in f32
    x = np.concatenate([x, 1.0 + (2 * np.arange(50) + 1) * 2.0 ** -8])   # bf16 ties
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.round_to(x, "bf16"), want)


def test_run_rounds_after_every_step():
    """run(round_fmt) == the single sweep (pinned above by FFT) rounded after every step."""
    dims = (6, 6)
    offs = oracle.offsets(2, "star", 1)
    c = np.full(len(offs), 0.2)
    for fmt in ("bf16", "f16", "f32"):
        x = oracle.round_to(inputs.uniform(121, dims), fmt)
        want = x.copy()
        for _ in range(4):
            want = oracle.round_to(oracle.sweep_const(want, offs, c, "dirichlet"), fmt)
        got = oracle.run(x, "const", "dirichlet", 4, offs=offs, coeffs=c, round_fmt=fmt)
        assert np.array_equal(got, want)
        assert np.array_equal(got, oracle.round_to(got, fmt))  # on the storage grid
        pure = oracle.run(x, "const", "dirichlet", 4, offs=offs, coeffs=c)
        assert not np.array_equal(got, pure)  # the rounding did happen


# --------------------------------------------------------------------------------------------
# wave equation, misfit and velocity gradient
# --------------------------------------------------------------------------------------------

def test_ricker_closed_form():
    f = 15.0
    dt = 1.0 / 15000.0  # t0 = 1/f falls on sample 1000
    w = inputs.ricker(f, dt, 2000)
    n0 = 1000
    assert abs(w[n0] - 1.0) < 1e-12 and np.argmax(w) == n0
    tz = 1.0 / (np.pi * f * np.sqrt(2.0))  # zero crossings at t0 +- tz
    z = inputs.ricker(f, 1.0, 1, t0=-tz)  # element 0 sits at tau = 0 - t0 = tz
    assert abs(z[0]) < 1e-12


def _small_wave(n=14, steps=40, seed=5901):
    v = inputs.velocity_field(seed, (n, n, n), width=3, passes=1)
    h = 10.0
    dt = 0.4 * h / 4500.0
    offs = oracle.offsets(3, "star", 4)
    c = inputs.laplacian_coeffs(offs, 4)
    wl = inputs.ricker(60.0, dt, steps)
    src = (n // 2, n // 2, n // 2)
    rz = 3
    return v, h, dt, offs, c, wl, src, rz, steps


def test_wave_first_steps_closed_form():
    v, h, dt, offs, c, wl, src, rz, _ = _small_wave()
    n = v.shape[0]
    _, u2 = oracle.wave_forward(v, offs, c, h, dt, 2, src, wl, rz, return_last=True)
    a = (v * dt / h) ** 2
    s0 = dt * dt * wl[0]
    s1 = dt * dt * wl[1]
    centre = c[[i for i, o in enumerate(offs) if not np.any(o)][0]]
    # u^1 = s0 e_src ;  u^2 = 2 u^1 + a (.) L u^1 + s1 e_src
    assert abs(u2[src] - (2 * s0 + a[src] * centre * s0 + s1)) < 1e-15 * abs(s0) * 100
    for o, w in zip(offs, c):
        if not np.any(o):
            continue
        p = tuple(s - int(d) for s, d in zip(src, o))  # cell whose tap o reads the source
        assert abs(u2[p] - a[p] * w * s0) <= 1e-13 * abs(a[p] * w * s0)
    assert u2[0, 0, 0] == 0.0 and n > 2


def test_wave_is_linear_in_the_source():
    v, h, dt, offs, c, wl, src, rz, steps = _small_wave(n=10, steps=12)
    t1 = oracle.wave_forward(v, offs, c, h, dt, steps, src, wl, rz)
    t2 = oracle.wave_forward(v, offs, c, h, dt, steps, src, 2.0 * wl, rz)
    assert relerr(t2, 2.0 * t1) < 1e-13


def test_misfit_closed_form():
    t = inputs.uniform(131, (3, 4, 5))
    o = inputs.uniform(132, (3, 4, 5))
    assert abs(oracle.misfit(t, o) - 0.5 * float(np.sum((t - o) ** 2))) < 1e-13


def test_gradient_checkpointed_equals_store_all_bitwise():
    v, h, dt, offs, c, wl, src, rz, steps = _small_wave(n=12, steps=30)
    obs = oracle.wave_forward(inputs.perturbed_velocity(v, sigma=3.0), offs, c, h, dt, steps,
                              src, wl, rz)
    J0, g0 = oracle.wave_gradient(v, offs, c, h, dt, steps, src, wl, rz, obs, ck_every=0)
    J1, g1 = oracle.wave_gradient(v, offs, c, h, dt, steps, src, wl, rz, obs, ck_every=7)
    assert J0 == J1 and np.array_equal(g0, g1)
    assert J0 == oracle.misfit(oracle.wave_forward(v, offs, c, h, dt, steps, src, wl, rz), obs)


def test_gradient_matches_finite_differences():
    v, h, dt, offs, c, wl, src, rz, steps = _small_wave(n=14, steps=40)
    obs = oracle.wave_forward(inputs.perturbed_velocity(v, sigma=3.0), offs, c, h, dt, steps,
                              src, wl, rz)
    J, g = oracle.wave_gradient(v, offs, c, h, dt, steps, src, wl, rz, obs, ck_every=10)
    e = inputs.box_mean_periodic(inputs.normal(5903, v.shape), 3)
    e /= np.max(np.abs(e))
    eps = 1e-2  # m/s on a field of ~3000 m/s
    jp = oracle.misfit(oracle.wave_forward(v + eps * e, offs, c, h, dt, steps, src, wl, rz), obs)
    jm = oracle.misfit(oracle.wave_forward(v - eps * e, offs, c, h, dt, steps, src, wl, rz), obs)
    fd = (jp - jm) / (2 * eps)
    ad = float(np.sum(g * e))
    assert J > 0 and abs(ad) > 0
    assert abs(fd - ad) <= 1e-6 * abs(ad)
