"""The oracle's Philox4x32-10 against the CUDA toolkit's own generator on the
GPU: cuRAND's device Philox4_32_10 with curand_init(seed, subsequence, 0)
yields, as its first four words, the Philox block of counter (0, 0,
subsequence low, subsequence high) under key (seed low, seed high).  The
library is run, not read: a small program calls curand_init / curand4 and
prints the words."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SRC = r"""
#include <cstdio>
#include <curand_kernel.h>
__global__ void k(const unsigned long long *seed, const unsigned long long *sub, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], sub[i], 0ull, &st);
    out[i] = curand4(&st);
}
int main() {
    const int n = 6;
    unsigned long long seed[n] = {0ull, 1ull, 0x123456789abcdefull, 0xffffffffffffffffull, 42ull, 7ull};
    unsigned long long sub[n] = {0ull, 5ull, 0xfedcba9876543210ull, 1ull << 40, 0x00000003ffffffffull, 123456789ull};
    unsigned long long *ds, *dq; uint4 *dout, out[n];
    cudaMalloc(&ds, sizeof(seed)); cudaMalloc(&dq, sizeof(sub)); cudaMalloc(&dout, sizeof(out));
    cudaMemcpy(ds, seed, sizeof(seed), cudaMemcpyHostToDevice);
    cudaMemcpy(dq, sub, sizeof(sub), cudaMemcpyHostToDevice);
    k<<<1, 32>>>(ds, dq, dout, n);
    if (cudaMemcpy(out, dout, sizeof(out), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    for (int i = 0; i < n; ++i)
        printf("%llu %llu %u %u %u %u\n", seed[i], sub[i], out[i].x, out[i].y, out[i].z, out[i].w);
    return 0;
}
"""


def test_oracle_philox_matches_curand(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "kat.cu"
    exe = tmp_path / "kat"
    src.write_text(SRC)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(int, line.split())) for line in out if line.strip()]
    assert len(rows) == 6
    for seed, sub, *words in rows:
        ctr = (0, 0, sub & 0xFFFFFFFF, sub >> 32)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), np.array(words, dtype=np.uint32),
                                      err_msg=f"seed {seed:#x} subsequence {sub:#x}")
