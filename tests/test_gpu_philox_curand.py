"""The device Philox4x32-10 that draws the pair noise (Groot-Warren random
force, counter-based generator of Salmon et al., SC'11) against cuRAND's
Philox4x32-10 and the oracle's, word for word, and its Box-Muller Gaussian
against the oracle's FP64 transform of the same words."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2512_13267_gb300 import build_ext

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("philox") / "philox_curand_check.so")
    cmd = [build_ext._nvcc()] + build_ext.NVCC_FLAGS + [
        "-shared", "-o", out, os.path.join(HERE, "philox_curand_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = C.CDLL(out)
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    lib.philox_curand_check.argtypes = [u32p, u32p, C.c_int, u32p, u32p, f32p]
    lib.philox_curand_check.restype = C.c_int
    return lib


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # the pair-noise shape: (min id, max id, step lo, step hi), key (seed lo, seed hi ^ box)
    ctr[:64, 0] = np.arange(64, dtype=np.uint32)
    ctr[:64, 1] = np.arange(64, dtype=np.uint32) + 1
    ctr[:64, 3] = 0
    ctr[64:72] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 0, 0, 0], [0, 0, 0, 1],
                  [0xFFFFFFFF, 0, 0, 0], [0, 0xFFFFFFFF, 0, 0], [0, 0, 0xFFFFFFFF, 0], [0, 0, 0, 0xFFFFFFFF]]
    key[64:72] = [[0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [1, 0], [0, 1],
                  [0x243F6A88, 0x85A308D3], [0, 0], [0, 0], [0, 0]]
    return np.ascontiguousarray(ctr), np.ascontiguousarray(key)


def test_device_philox_words_equal_curand_and_oracle(harness, parity_report):
    n = 4096
    ctr, key = _inputs(n, 5)
    mine = np.zeros((n, 2), np.uint32)
    ref = np.zeros((n, 4), np.uint32)
    theta = np.zeros(n, np.float32)
    assert harness.philox_curand_check(ctr.ravel(), key.ravel(), n, mine.ravel(), ref.ravel(),
                                       theta) == 0
    # bit for bit: the library's two words are cuRAND's first two
    assert np.array_equal(mine, ref[:, :2])
    # and the oracle's (all four words) on a sample
    for t in range(0, n, 37):
        assert O.philox4x32_10(ctr[t].tolist(), key[t].tolist()) == ref[t].tolist()
    # FP32 Box-Muller of the same words against the oracle's FP64 transform.
    # Error budget of the FP32 path: ln u1 and the square root to < 1e-6
    # relative, the hardware cosine (with the FP32 2 pi) to < 1e-6 absolute,
    # so |dtheta| < 1e-6 (r + |theta|) with r = sqrt(-2 ln u1); the test
    # allows twice that.
    exp = np.array([O.theta_from_words(int(a), int(b)) for a, b in mine])
    u1 = ((mine[:, 0] >> 9).astype(np.float64) + 0.5) * 2.0**-23
    scale = np.sqrt(-2.0 * np.log(u1)) + np.abs(exp)
    rel = np.abs(theta.astype(np.float64) - exp) / scale
    parity_report("Box-Muller theta from the pair words (FP32 device)", float(rel.max()), 2e-6,
                  "max |dtheta| / (r + |theta|)")
    assert rel.max() <= 2e-6, float(rel.max())
    # the words are well spread: the Gaussian sample has the right moments
    assert abs(exp.mean()) < 4.0 / np.sqrt(n) and abs(exp.var() - 1.0) < 6.0 * np.sqrt(2.0 / n)
