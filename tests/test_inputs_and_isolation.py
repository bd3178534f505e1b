"""The seeded input generators, and the separation between the product, the
oracle and the inputs (CPU only).

- The generators are reproducible and have the stated structure: points on
  the unit sphere or the ellipsoid, N(0, 1) right-hand sides, and batch
  specs within their ranges.
- The product package and the CUDA sources never reach the oracle.
- The oracle never reaches the product package.
- The generators import neither of them."""
import ast
import math
import os

import numpy as np

from workloads import CONFIGS, batch_specs, ellipsoid_points, gaussian_rhs, sphere_points

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sphere_and_ellipsoid_points():
    p = sphere_points(5000, 3)
    assert p.shape == (5000, 3) and p.dtype == np.float64 and p.flags.c_contiguous
    np.testing.assert_allclose(np.linalg.norm(p, axis=1), 1.0, rtol=0, atol=1e-15)
    assert np.array_equal(p, sphere_points(5000, 3))
    assert not np.array_equal(p, sphere_points(5000, 4))
    # uniform on S²: each coordinate has mean 0 and variance 1/3
    assert np.all(np.abs(p.mean(axis=0)) < 0.05)
    np.testing.assert_allclose(p.var(axis=0), 1.0 / 3.0, atol=0.02)
    axes = (0.6, 1.9, 1.2)
    e = ellipsoid_points(5000, axes, 3)
    np.testing.assert_allclose(((e / np.asarray(axes)) ** 2).sum(axis=1), 1.0, atol=1e-14)


def test_gaussian_rhs():
    x = gaussian_rhs(20000, 8, 5)
    assert x.shape == (20000, 8) and x.flags.c_contiguous
    assert abs(x.mean()) < 0.02 and abs(x.std() - 1.0) < 0.02
    assert np.array_equal(x, gaussian_rhs(20000, 8, 5))


def test_batch_specs_ranges():
    specs = batch_specs()
    assert len(specs) == 64
    for s in specs:
        assert 2048 <= s["n"] <= 32768 and 1 <= s["m"] <= 64 and s["q"] in (3, 4)
        assert all(0.5 <= a <= 2.0 for a in s["axes"])
    assert len({s["point_seed"] for s in specs}) == 64
    # log-uniform n: the median sits near the geometric mean of the range
    med = np.median([s["n"] for s in specs])
    assert 0.5 * math.sqrt(2048 * 32768) < med < 2.0 * math.sqrt(2048 * 32768)
    assert CONFIGS["precision_n65536"]["n"] == 65536 and CONFIGS["precision_n65536"]["q"] == 4


def _imports(path):
    tree = ast.parse(open(path, encoding="utf-8").read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            if node.level:
                names.add("." + (node.module or ""))
            elif node.module:
                names.add(node.module.split(".")[0])
    return names


def _py_files(folder):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def test_product_never_reaches_the_oracle():
    for path in _py_files("paper_2509_17257_gb300"):
        assert "oracle" not in _imports(path), path
    csrc = os.path.join(ROOT, "paper_2509_17257_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f), encoding="utf-8").read()
        assert "oracle/" not in text and "h2_oracle" not in text, f


def test_oracle_and_inputs_never_reach_the_product():
    for folder in ("oracle", "workloads"):
        for path in _py_files(folder):
            imps = _imports(path)
            assert "paper_2509_17257_gb300" not in imps, path
            if folder == "workloads":
                assert "oracle" not in imps, path
