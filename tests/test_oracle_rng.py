"""Pins of the oracle's counter-based generator (no GPU).

The oracle's Philox4x32-10 is compared with an independent implementation,
PyTorch's at::philox_engine, compiled from the installed ATen header."""
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import stats

HERE = os.path.dirname(os.path.abspath(__file__))


def _aten_philox():
    try:
        import torch
    except ImportError:
        pytest.skip("torch headers not available")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    if not os.path.exists(hdr) or shutil.which("g++") is None:
        pytest.skip("ATen Philox header or g++ missing")
    exe = os.path.join(HERE, "pins", f"philox_aten.{os.uname().machine}.bin")
    src = os.path.join(HERE, "pins", "philox_aten.cpp")
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.run(["g++", "-O1", "-std=c++17", "-I" + inc, src, "-o", exe], check=True)
    return exe


def test_philox_matches_aten_engine(O):
    exe = _aten_philox()
    rng = np.random.default_rng(12345)
    ctr = rng.integers(0, 2 ** 32, size=(2000, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    lines = "\n".join(" ".join("%x" % v for v in list(c) + list(k)) for c, k in zip(ctr, key)) + "\n"
    out = subprocess.run([exe], input=lines, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(t, 16) for t in ln.split()] for ln in out.strip().splitlines()], np.uint32)
    got = O.philox(ctr, key)
    assert np.array_equal(got, ref)


def test_uniform_lattice(O):
    r = np.array([0, 1, 255, 256, 0x7FFFFFFF, 0x80000000, 0xFFFFFF00, 0xFFFFFFFF], np.uint32)
    u = O.uniform(r)
    assert u[0] == 2.0 ** -24 and u[-1] == 1.0 - 2.0 ** -24
    assert np.all((u > 0) & (u < 1))
    k = u * 2 ** 24
    assert np.all(k == np.round(k)) and np.all(np.round(k) % 2 == 1)
    # symmetric under u -> 1 - u: r and ~r map to mirror images
    assert np.allclose(O.uniform(~r) + u, 1.0, rtol=0, atol=0)


def test_philox_stream_is_uniform(O):
    n = 200000
    ctr = np.zeros((n // 4, 4), np.uint32)
    ctr[:, 0] = np.arange(n // 4)
    ctr[:, 2] = 7
    r = O.philox(ctr, np.array([1, 0], np.uint32)).ravel()
    counts = np.bincount(r >> 24, minlength=256)
    assert stats.chisquare(counts).pvalue > 1e-3
    u = (r.astype(np.float64) + 0.5) / 2 ** 32
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01
