"""The integer slice split of the tensor-core FP64 product (csrc/ozaki_split.cuh) against the
oracle's FP64 split (oracle/ozaki.py), bit for bit, on the host: column exponents and every
digit, for random columns, ties at every slice, values far below the column maximum, and zero
and power-of-two columns. A host program built with nvcc does the comparison (no GPU)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import ozaki


def _nvcc():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    return nvcc


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    src = os.path.join(os.path.dirname(__file__), "native", "ozaki_split_check.cu")
    exe = str(tmp_path_factory.mktemp("oz") / "ozaki_split_check")
    subprocess.run([_nvcc(), "-O2", "-std=c++17", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    return exe


def _columns(rng, d):
    cols = []
    # mixed magnitudes and signs
    for e in (-40, -7, 0, 3, 60, 150):
        cols.append(rng.standard_normal(d) * 2.0 ** e)
    # values spread over 60 binades below the column maximum (deep residual bits, sticky bits)
    c = rng.standard_normal(d) * np.ldexp(1.0, rng.integers(-60, 1, size=d))
    c[0] = 1.0
    cols.append(c)
    # exact ties at slice boundaries: multiples of half units for beta = 9, E = 0
    units = [2.0 ** (0 - 8 - 9 * k) for k in range(6)]
    t = np.zeros(d)
    for r in range(d):
        k = r % 6
        t[r] = (rng.integers(-200, 200) + 0.5) * units[k] * (1 if r % 2 else -1)
    t[0] = 1.0
    cols.append(t)
    # zero column and a power-of-two maximum
    cols.append(np.zeros(d))
    p = rng.standard_normal(d) * 0.25
    p[3] = -2.0
    cols.append(p)
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("beta,s", [(9, 6), (8, 7), (7, 8), (5, 3)])
def test_integer_slices_match_oracle_bit_for_bit(checker, tmp_path, beta, s):
    rng = np.random.default_rng(1000 + beta)
    X = _columns(rng, 257)
    a, u, _ = ozaki.split(X, beta, s)
    E = ozaki.column_exponents(X)
    path = tmp_path / "case.bin"
    with open(path, "wb") as f:
        np.array([X.shape[0], X.shape[1], beta, s], dtype=np.int32).tofile(f)
        np.asfortranarray(X).ravel(order="F").astype(np.float64).tofile(f)
        E.astype(np.int64).tofile(f)
        a.astype(np.int64).tofile(f)
    r = subprocess.run([checker, str(path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.fixture(scope="module")
def gram_checker(tmp_path_factory):
    src = os.path.join(os.path.dirname(__file__), "native", "ozaki_gram_check.cu")
    exe = str(tmp_path_factory.mktemp("ozg") / "ozaki_gram_check")
    subprocess.run([_nvcc(), "-O2", "-std=c++17", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    return exe


@pytest.mark.parametrize("beta,s", [(9, 6), (8, 7)])
def test_slice_product_pipeline_matches_oracle_gram_bit_for_bit(gram_checker, tmp_path, beta,
                                                                 s):
    """Split, exact integer sums of the slice products on each diagonal and oz_combine
    reproduce oracle.gram exactly: the only rounding is the single rounding of the exact sum."""
    rng = np.random.default_rng(77 + beta)
    A = _columns(rng, 300)
    B = _columns(rng, 300)[:, ::-1].copy()
    B[:, 1] = A[:, 2]  # a shared column (a Gram diagonal entry)
    C = ozaki.gram(A, B, beta, s)
    path = tmp_path / "gram.bin"
    with open(path, "wb") as f:
        np.array([A.shape[0], A.shape[1], B.shape[1], beta, s], dtype=np.int32).tofile(f)
        A.ravel(order="F").astype(np.float64).tofile(f)
        B.ravel(order="F").astype(np.float64).tofile(f)
        np.ascontiguousarray(C).astype(np.float64).tofile(f)
    r = subprocess.run([gram_checker, str(path)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.fixture(scope="module")
def plan_checker(tmp_path_factory):
    src = os.path.join(os.path.dirname(__file__), "native", "ozaki_plan_check.cu")
    exe = str(tmp_path_factory.mktemp("ozp") / "ozaki_plan_check")
    subprocess.run([_nvcc(), "-O2", "-std=c++17", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    return exe


def _run_plan(plan_checker, tmp_path, A, B, beta, s, chunk):
    C = ozaki.gram(A, B, beta, s)
    path = tmp_path / "plan.bin"
    with open(path, "wb") as f:
        np.array([A.shape[0], A.shape[1], B.shape[1], beta, s, chunk], dtype=np.int32).tofile(f)
        A.ravel(order="F").astype(np.float64).tofile(f)
        B.ravel(order="F").astype(np.float64).tofile(f)
        np.ascontiguousarray(C).astype(np.float64).tofile(f)
    return subprocess.run([plan_checker, str(path)], capture_output=True, text=True, timeout=600)


def test_chunked_slice_product_plan_is_exact_and_matches_oracle(plan_checker, tmp_path):
    """The kernel's layout, beta = 7 and s = 8 with one FP32 accumulator per diagonal
    k + l = t over windows of 512 rows (the exactness length for up to 8 pairs of products of
    at most 2^12), reproduces oracle.gram bit for bit over 9000 rows (18 windows, the last
    ragged), with the magnitudes of every window's products within 2^24."""
    win = ozaki.max_exact_diagonal_window(7, 8)
    assert win == 512
    rng = np.random.default_rng(4096)
    A = _columns(rng, 9000)[:, :6]
    B = _columns(rng, 9000)[:, 2:8].copy()
    B[:, 0] = A[:, 1]
    r = _run_plan(plan_checker, tmp_path, A, B, 7, 8, win)
    assert r.returncode == 0, r.stdout[-2000:]
    W = np.full((9000, 2), 1.0)
    r = _run_plan(plan_checker, tmp_path, W, W, 7, 8, win)
    assert r.returncode == 0, r.stdout[-2000:]


def test_chunk_past_the_exactness_length_is_flagged(plan_checker, tmp_path):
    """Columns of ones have a leading slice of 64 in every row: 4096 rows of products 2^12
    reach 2^24, so a window of 8192 rows is flagged, as it must be."""
    W = np.full((9000, 2), 1.0)
    r = _run_plan(plan_checker, tmp_path, W, W, 7, 8, 8192)
    assert r.returncode != 0 and "beyond 2^24" in r.stdout
    r = _run_plan(plan_checker, tmp_path, W, W, 7, 8, 4096)
    assert r.returncode == 0, r.stdout[-2000:]
