"""Device Philox4x32-10 against the oracle's (bit-exact) and against cuRAND's
Philox4_32_10, an independent implementation of the same published
generator (GPU)."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import philox as orc_philox

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def dsmc():
    import __graft_entry__ as g
    g.build()
    from paper_cs_9902024_gb300 import dsmc as D
    return D


def test_device_philox_equals_oracle(dsmc):
    rng = np.random.default_rng(11)
    n = 4096
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    out = dsmc.philox_gpu(ctr, key)
    ref = np.array([orc_philox(ctr[i], key[i]) for i in range(n)])
    assert np.array_equal(out, ref)


def test_device_philox_equals_curand(dsmc):
    with tempfile.TemporaryDirectory() as d:
        so = os.path.join(d, "curand_ref.so")
        subprocess.check_call(["/usr/local/cuda/bin/nvcc", "-shared", "-Xcompiler", "-fPIC",
                               "-gencode", "arch=compute_103a,code=sm_103a",
                               os.path.join(HERE, "gpu_curand_ref.cu"), "-o", so])
        lib = C.CDLL(so)
        rng = np.random.default_rng(12)
        n = 2048
        seed = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
        sub = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
        cc = rng.integers(0, 2 ** 40, n, dtype=np.uint64)
        out = np.zeros((n, 4), dtype=np.uint32)
        P = C.POINTER(C.c_ulonglong)
        rc = lib.curand_philox_ref(n, seed.ctypes.data_as(P), sub.ctypes.data_as(P),
                                   cc.ctypes.data_as(P), out.ctypes.data_as(C.POINTER(C.c_uint)))
        assert rc == 0
    ctr = np.stack([cc & 0xFFFFFFFF, cc >> 32, sub & 0xFFFFFFFF, sub >> 32], 1).astype(np.uint32)
    key = np.stack([seed & 0xFFFFFFFF, seed >> 32], 1).astype(np.uint32)
    mine = dsmc.philox_gpu(ctr, key)
    assert np.array_equal(mine, out)
