"""Pin the oracle's Philox4x32-10 against an independent implementation.

The paper names no random number generator; the build uses the counter-based Philox4x32-10 of
Salmon et al. (SC'11).  The oracle's copy is checked block by block against PyTorch's
header-only CPU Philox engine (ATen/core/PhiloxRNGEngine.h), compiled here with g++.  That
engine maps (seed, subsequence, offset) to key (seed_lo, seed_hi) and counter
(offset_lo, offset_hi, subsequence_lo, subsequence_hi), so any counter/key pair can be driven.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch_include():
    try:
        import torch  # noqa: F401
        inc = os.path.join(os.path.dirname(torch.__file__), "include")
    except Exception:
        return None
    return inc if os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")) else None


@pytest.fixture(scope="module")
def aten_philox(tmp_path_factory):
    inc = _torch_include()
    if inc is None or shutil.which("g++") is None:
        pytest.skip("PyTorch headers or g++ not available")
    exe = str(tmp_path_factory.mktemp("philox") / "aten_philox")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, "-o", exe,
                    os.path.join(HERE, "philox_aten_harness.cpp")], check=True)

    def run(rows):
        text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)
    return run


def test_philox_matches_aten_engine(aten_philox):
    rng = np.random.default_rng(12345)
    rows = rng.integers(0, 2**32, size=(1500, 6), dtype=np.uint64)
    edge = [0, 1, 0xFFFFFFFF, 0x80000000]
    extra = np.array([[a, b, c, d, e, f] for a in edge for b in edge[:2] for c in edge
                      for d in edge[:2] for e in edge[:2] for f in edge[::3]], dtype=np.uint64)
    rows = np.concatenate([rows, extra])
    want = aten_philox(rows)
    got = np.array([oracle.philox4x32_10(r[:4], r[4:]) for r in rows], dtype=np.uint64)
    assert np.array_equal(got, want)


def test_philox_counter_layout_used_by_dynamics(aten_philox):
    """The dynamics key by (vertex, sweep, replica/4, domain); check such counters too."""
    rows = []
    for i in (0, 1, 1023, 2**22 - 1):
        for t in (0, 1, 65535):
            for z in (0, 1, 63):
                for dom in (0, 1):
                    rows.append([i, t, z, dom, 1, 0])
    rows = np.array(rows, dtype=np.uint64)
    want = aten_philox(rows)
    got = np.array([oracle.philox4x32_10(r[:4], r[4:]) for r in rows], dtype=np.uint64)
    assert np.array_equal(got, want)


def test_philox_words_look_uniform():
    """Coarse sanity: byte histogram of 4096 blocks is flat (chi-square, 255 dof)."""
    words = np.array([oracle.philox4x32_10([i, 7, 3, 0], [1, 0]) for i in range(4096)],
                     dtype=np.uint32)
    b = words.view(np.uint8).ravel()
    hist = np.bincount(b, minlength=256).astype(float)
    exp = b.size / 256.0
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert 150 < chi2 < 380
