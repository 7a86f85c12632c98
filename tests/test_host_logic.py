"""Host-side checks that need no GPU: the product path never touches the oracle, fails
loudly without its shared library, and the seeded input recipes are deterministic and
inside the domains they claim."""
import ast
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2605_15547_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom):
            yield node.module or ""


def test_product_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith(".py"):
                mods = list(_imports(os.path.join(dirpath, f)))
                assert not any(m == "oracle" or m.startswith("oracle.") for m in mods), f


def test_cuda_sources_never_include_the_oracle():
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f), errors="replace").read()
        assert "crm_oracle" not in text and "oracle/" not in text, f


def test_missing_library_raises(monkeypatch):
    from paper_2605_15547_gb300 import _lib as L
    monkeypatch.setattr(L, "LIB_PATH", os.path.join(PKG, "no_such_library.so"))
    monkeypatch.setattr(L, "_LIB", None)
    with pytest.raises(ImportError):
        L.lib()


def test_recipes_are_deterministic():
    from paper_2605_15547_gb300 import workloads as W
    for wl in ("all19", "precision", "trig", "f64"):
        arrays, cfg = W.bench_arrays(wl, scale=14)
        assert cfg["workload"]
        for label, func, n in arrays:
            a = W.bench_input_host(wl, label, func, n)
            b = W.bench_input_host(wl, label, func, n)
            assert a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8)), label


def test_domain_recipe_stays_inside_the_domain():
    from paper_2605_15547_gb300 import workloads as W
    rng = np.random.default_rng(0)
    for func in W.F32_FUNCS:
        x = W.domain_bits(func, 20000, rng, special_frac=0.0).view(np.float32)
        lo, hi = W.DOMAIN_F32[func]
        assert np.all(np.isfinite(x)) and np.all(x > lo) and np.all(x < hi), func


def test_bench_sizes_match_the_stated_workloads():
    from paper_2605_15547_gb300 import workloads as W
    arrays, _ = W.bench_arrays("all19")
    assert len(arrays) == 19 and all(n == 1 << 26 for _, _, n in arrays)
    arrays, _ = W.bench_arrays("precision")
    assert len(arrays) == 11 and all(n == 1 << 28 for _, _, n in arrays)
    rng = np.random.Generator(np.random.PCG64(W.seed_for(4, 0)))
    lens, funcs = W.batch_lengths(10000, rng)
    assert lens.min() >= 64 and lens.max() <= 1 << 22 and 3.5e9 < lens.sum() < 4.1e9
    assert set(funcs) <= set(W.F32_FUNCS)


def test_near_multiples_of_pio2_are_near():
    from paper_2605_15547_gb300 import workloads as W
    x = W.near_multiples_of_pio2(2000, np.random.default_rng(1)).astype(np.float64)
    k = np.round(np.abs(x) / (np.pi / 2))
    rel = np.abs(np.abs(x) - k * np.pi / 2) / np.maximum(k, 1)
    assert np.median(rel) < 1e-4
