"""The oracle's Philox-4x32-10 against cuRAND's (GPU required).

The samplers' counters go through Philox-4x32-10 (Salmon et al., SC'11),
which the oracle implements from the published definition.  cuRAND ships
the same round function (curand_Philox4x32_10 in its device headers); a
small kernel here calls it on random counters and keys, and every output
word must equal the oracle's.  With the Triton pin on the CPU this pins the
oracle's Philox to two independent implementations.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    out = os.path.join(tempfile.mkdtemp(), "libcurand_philox_ref.so")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                    "-Xcompiler", "-fPIC", os.path.join(HERE, "curand_philox_ref.cu"), "-o", out],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    lib.curand_philox_batch.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    return lib


def test_oracle_philox_equals_curand(curand_lib):
    rng = np.random.default_rng(31)
    n = 4096
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [5, 0, 7, 2]]   # edge counters
    key[:4] = [[0, 0], [0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [5, 6]]
    d_ctr = torch.from_numpy(ctr.view(np.int32)).cuda()
    d_key = torch.from_numpy(key.view(np.int32)).cuda()
    d_out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    assert curand_lib.curand_philox_batch(ctypes.c_void_p(d_ctr.data_ptr()),
                                          ctypes.c_void_p(d_key.data_ptr()),
                                          ctypes.c_void_p(d_out.data_ptr()), n) == 0
    got = d_out.cpu().numpy().view(np.uint32)
    for i in range(n):
        want = oracle.philox(ctr[i].tolist(), key[i].tolist())
        assert np.array_equal(got[i], np.asarray(want, np.uint32)), i
