"""The oracle's Philox4x32-10 (the noise of the Langevin thermostat, Sec.
III.A) pinned to an implementation written elsewhere: NVIDIA's cuRAND
Philox4_32_10, run through its public device API in a test-only kernel
(tests/philox_curand.cu), must give the oracle's words bit for bit on more
than a million counters -- random 128-bit counters and keys, and the
counter layout the library uses, (atom, step_lo, step_hi, replica << 4 |
stream).  A swapped multiplier, word order or key increment in the oracle
fails it.  The library's own noise (ne_noise) is then compared with the
oracle's normals over as many counters."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2201_04622_gb300 import ne  # noqa: E402

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
N_CTR = 1 << 20


@pytest.fixture(scope="module")
def curand_lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp(prefix="curand_philox_")
    so = os.path.join(d, "libcurand_philox.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", so, os.path.join(HERE, "philox_curand.cu")])
    L = C.CDLL(so)
    L.curand_philox_blocks.argtypes = [C.c_ulonglong, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    L.curand_philox_blocks.restype = C.c_int
    yield L
    shutil.rmtree(d, ignore_errors=True)


def curand_blocks(L, seed, ctr):
    dev = torch.device("cuda:0")
    c = torch.from_numpy(np.ascontiguousarray(ctr, dtype=np.uint32).view(np.int32)).to(dev)
    out = torch.zeros_like(c)
    st = torch.cuda.current_stream().cuda_stream
    assert L.curand_philox_blocks(int(seed), c.data_ptr(), c.shape[0], out.data_ptr(), st) == 0
    return out.cpu().numpy().view(np.uint32)


def test_oracle_philox_equals_curand_on_random_counters(curand_lib):
    rng = np.random.default_rng(2201)
    for seed in [0, 1, 2 ** 40 + 5, int(rng.integers(0, 2 ** 63))]:
        ctr = rng.integers(0, 2 ** 32, size=(N_CTR // 4, 4), dtype=np.uint64).astype(np.uint32)
        ctr[:8] = [[0, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1],
                   [0xFFFFFFFF] * 4, [0xFFFFFFFF, 0xFFFFFFFF, 0, 0], [0, 0, 0xFFFFFFFF, 0xFFFFFFFF]]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = curand_blocks(curand_lib, seed, ctr)
        want = O.philox_many(ctr, key)
        assert np.array_equal(got, want), (seed, np.argwhere(got != want)[:4])


def test_oracle_philox_equals_curand_on_the_noise_counters(curand_lib):
    """(atom, step_lo, step_hi, replica << 4 | stream) for 2^18 atoms at four
    (seed, replica, stream, step) of the kind the runs use."""
    n = N_CTR // 4
    atoms = np.arange(n, dtype=np.uint64)
    for seed, rep, stream, step in [(1, 0, 0, 0), (7, 3, 2, 123456), (2 ** 40 + 5, 17, 4, 2 ** 33 + 9),
                                    (10, (1 << 28) - 1, 5, 2 ** 32 - 1)]:
        ctr = np.stack([atoms, np.full(n, step & 0xFFFFFFFF), np.full(n, step >> 32),
                        np.full(n, (rep << 4) | stream)], axis=1).astype(np.uint32)
        got = curand_blocks(curand_lib, seed, ctr)
        want = O.philox_many(ctr, [seed & 0xFFFFFFFF, seed >> 32])
        assert np.array_equal(got, want), (seed, rep, stream, step)


def test_library_noise_matches_oracle_normals_on_a_million_counters():
    """ne_noise (FP64) against the oracle's Box-Muller normals of the same
    Philox blocks: 2^20 atoms at each of two (seed, replica, stream, step)."""
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    dev = torch.device("cuda:0")
    n = N_CTR
    for seed, rep, stream, step in [(3, 5, 0, 98765), (2 ** 33 + 1, 200, 4, 2 ** 32 + 17)]:
        z = torch.zeros((n, 3), dtype=torch.float64, device=dev)
        ne.ne_noise(seed, rep, stream, step, z, ne.NE_FP64)
        zo = O.normals_many(seed, rep, stream, step, n)
        # libm vs CUDA log/sincospi differ in the last bits only; a different
        # Philox word moves a normal by O(1)
        assert np.abs(z.cpu().numpy() - zo).max() < 1e-12
