"""Pins of the BF16 error budget (oracle ``round_bf16`` and ``h2mm_bf16``):
the product with operands rounded to bfloat16 and FP32 accumulation, used to
predict the error of the BF16 tensor-core product.

* rounding: values worked out by hand (ties to even, a carry, one rounding
  from FP64), the unit roundoff 2^-8 of 8 significant bits as the bound of
  the relative error and that it is attained, and torch's own
  float32 -> bfloat16 conversion;
* the product: without rounding it is the FP32 product; rounding one operand
  equals the FP64 product of a matrix whose operand was rounded beforehand;
  with dyadic data every step is exact and the result is the FP64 product
  bit for bit."""
import copy

import numpy as np
import pytest

from _helpers import rel_fro
from oracle import h2_oracle as O
from workloads import gaussian_rhs, sphere_points


def test_round_bf16_hand_values():
    u = 2.0 ** -8
    cases = {
        1.0: 1.0,
        1.0 + u: 1.0,                      # halfway between 1 and 1 + 2^-7: tie to the even 1.0
        1.0 + 3 * u: 1.0 + 4 * u,          # halfway between 1 + 2^-7 and 1 + 2^-6: tie to the even 1 + 2^-6
        1.0 + u + 2.0 ** -30: 1.0 + 2 * u, # just above the midpoint: up (an FP32 step first would give 1.0)
        1.0 / 3.0: 0.333984375,            # 1.0101010|101... x 2^-2 rounds up to 1.0101011 x 2^-2
        -2.75: -2.75,                      # representable
        255.5: 256.0,                      # 8 significant bits: 255.5 is a tie, 256 the even neighbour
        0.0: 0.0,
        2.0 ** 100 * (1 + 2 * u): 2.0 ** 100 * (1 + 2 * u),
    }
    got = O.round_bf16(np.array(list(cases)))
    assert np.array_equal(got, np.array(list(cases.values())))


def test_round_bf16_error_bound_is_attained():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-20, 20, 200000))
    r = O.round_bf16(x)
    rel = np.abs(r - x) / np.abs(x)
    # 8 significant bits: unit roundoff u = 2^-8, reached just above a power of two
    assert rel.max() <= 2.0 ** -8
    assert rel.max() >= 0.99 * 2.0 ** -8  # round to nearest: a cut after 8 bits would reach 2^-7
    # the result has at most 8 significant bits
    f, _ = np.frexp(r)
    assert np.all(np.ldexp(f, 8) == np.rint(np.ldexp(f, 8)))


def test_round_bf16_matches_torch_on_fp32_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-30, 30, 100000))).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x.astype(np.float64)), want)


@pytest.fixture(scope="module")
def case():
    pts = sphere_points(2048, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    X = gaussian_rhs(2048, 5, 1)
    Y0 = gaussian_rhs(2048, 5, 2)
    return H, X, Y0


def test_without_rounding_it_is_the_fp32_product(case):
    H, X, Y0 = case
    want = O.h2mm(H, 0.75, X, Y0)
    got = O.h2mm_bf16(H, 0.75, X, Y0, rounded=())
    assert rel_fro(got, want) <= 2e-6
    gotT = O.h2mm_bf16(H, 0.75, X, Y0, rounded=(), transposed=True)
    assert rel_fro(gotT, O.h2mm(H, 0.75, X, Y0, transposed=True)) <= 2e-6


def _rounded_copy(H, name):
    """A copy of H whose operand `name` is rounded to BF16 beforehand (FP64 storage)."""
    R = copy.copy(H)
    if name in ("Vf", "Vb", "V"):
        R.V = {i: O.round_bf16(v) for i, v in H.V.items()}
    elif name == "E":
        R.E = {i: O.round_bf16(e) for i, e in H.E.items()}
    elif name in ("S", "G"):
        blocks = [copy.copy(b) for b in (H.adm if name == "S" else H.near)]
        for b in blocks:
            if name == "S":
                b.S = O.round_bf16(b.S)
            else:
                b.G = O.round_bf16(b.G)
        R.btree = _replace_leaves(H.btree, {id(o): b for o, b in zip(H.adm if name == "S" else H.near, blocks)})
        if name == "S":
            R.adm = blocks
        else:
            R.near = blocks
    return R


def _replace_leaves(b, repl):
    if id(b) in repl:
        return repl[id(b)]
    if not b.sons:
        return b
    c = copy.copy(b)
    c.sons = [_replace_leaves(s, repl) for s in b.sons]
    return c


@pytest.mark.parametrize("name", ["V", "E", "S", "G"])
@pytest.mark.parametrize("transposed", [False, True])
def test_rounding_one_operand_equals_a_matrix_built_with_it_rounded(case, name, transposed):
    H, X, Y0 = case
    exact = O.h2mm(H, 0.75, X, Y0, transposed=transposed)
    want = O.h2mm(_rounded_copy(H, name), 0.75, X, Y0, transposed=transposed)
    got = O.h2mm_bf16(H, 0.75, X, Y0, rounded=(name,), transposed=transposed)
    effect = rel_fro(want, exact)
    assert 1e-5 <= effect <= 2.0 ** -8  # the rounding changes the product, at the BF16 level
    assert rel_fro(got, want) <= 2e-6   # and the emulation applies it where the matrix holds it


def test_rounding_x_rounds_the_block_product_but_not_the_shift(case):
    H, X, Y0 = case
    Xr = O.round_bf16(X)
    want = O.h2mm(H, 0.75, Xr, Y0) + 0.75 * H.sigma * (X - Xr)
    got = O.h2mm_bf16(H, 0.75, X, Y0, rounded=("X",))
    assert rel_fro(got, want) <= 2e-6


def test_forward_and_backward_bases_split_the_v_rounding(case):
    """Rounding V in the forward and in the backward transformation are two
    separate first-order perturbations that add up to rounding V in both."""
    H, X, Y0 = case
    base = O.h2mm_bf16(H, 1.0, X, rounded=())
    d_f = O.h2mm_bf16(H, 1.0, X, rounded=("Vf",)) - base
    d_b = O.h2mm_bf16(H, 1.0, X, rounded=("Vb",)) - base
    d_v = O.h2mm_bf16(H, 1.0, X, rounded=("V",)) - base
    assert np.linalg.norm(d_f) > 0 and np.linalg.norm(d_b) > 0
    assert np.linalg.norm(d_f + d_b - d_v) <= 2e-2 * np.linalg.norm(d_v)


def test_dyadic_single_block_is_exact():
    """n <= leaf size: one nearfield block.  Kernel values 1/2 and 1, integer
    X, sigma = 1/4: every operand is a BF16 value and every FP32 sum is exact,
    so the emulated product equals the FP64 product bit for bit."""
    rng = np.random.default_rng(7)
    pts = rng.uniform(0.0, 1.0, size=(24, 3))

    def g(x, y):
        d = x - y
        return np.where((d * d).sum(axis=-1) > 0.25, 0.5, 1.0)

    H = O.H2Matrix(pts, q=2, leaf_size=64, eta=2.0, kernel=g, sigma=0.25)
    X = rng.integers(-8, 9, size=(24, 3)).astype(np.float64)
    Y0 = rng.integers(-8, 9, size=(24, 3)).astype(np.float64)
    want = O.h2mm(H, 2.0, X, Y0)
    got = O.h2mm_bf16(H, 2.0, X, Y0)
    assert np.array_equal(got, want)
    assert np.array_equal(got, Y0 + 2.0 * (g(pts[:, None, :], pts[None, :, :]) @ X + 0.25 * X))


def test_budget_magnitude_at_the_bf16_level():
    """All operands rounded: the relative error is of the order of the BF16
    unit roundoff 2^-8 (not the FP32 one, not a lost term)."""
    pts = sphere_points(4096, 0)
    H = O.H2Matrix(pts, q=3, leaf_size=64, eta=2.0, sigma=1e-2)
    X = gaussian_rhs(4096, 4, 1)
    err = rel_fro(O.h2mm_bf16(H, 1.0, X), O.h2mm(H, 1.0, X))
    assert 0.05 * 2.0 ** -8 <= err <= 2 * 2.0 ** -8, err
