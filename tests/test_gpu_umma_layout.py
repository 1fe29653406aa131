"""Pins the tcgen05 shared-memory descriptor fields used by the tensor-core kernels: one MMA chain
D = A B^T (M = 128, K = 128, BF16 in, FP32 out) on host-prepared operand images, compared exactly with
numpy (small integers, exact in BF16 and FP32).

K-major image of a [R][K] tile: element (r, k) at (r/8)*16K + (k/8)*128 + (r%8)*16 + (k%8)*2, read
with LBO = 128 (next 8 k) and SBO = 16K (next 8 rows), start += 256 per 16-k step.
MN-major use of the same bytes: the stored [K'][M'] tile is the operand A[m][k] = T[k][m]; its 8-element
MN groups are 128 B apart and its 8-row K groups 16 M' B apart.
8-bit (E4M3, kind::f8f6f4) K-major image: element (r, k) at (r/8)*8K + (k/16)*128 + (r%8)*16 + k%16, read
with LBO = 128 and SBO = 8K, start += 256 per 32-k step."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def canon_image(T):
    """Byte image (as uint16 array) of a [R][K] tile in the canonical K-major layout."""
    R, K = T.shape
    img = np.zeros(R * K, dtype=np.uint16)
    r, k = np.meshgrid(np.arange(R), np.arange(K), indexing="ij")
    off = ((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2) // 2
    bits = torch.as_tensor(T.astype(np.float32)).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    img[off.reshape(-1)] = bits.reshape(-1)
    return img


@pytest.fixture(scope="module")
def probe():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = os.path.join(HERE, "_build")
    os.makedirs(out, exist_ok=True)
    so = os.path.join(out, "umma_probe.so")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-shared", os.path.join(HERE, "cuda", "umma_probe.cu"), "-o", so], check=True)
    L = C.CDLL(so)
    L.umma_probe_run.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int] + \
                                [C.c_uint32] * 6 + [C.c_int, C.c_void_p, C.c_void_p]
    return L


def run(L, a_img, b_img, N, a_mn, b_mn, a_fields, b_fields, f8=0):
    A = torch.as_tensor(a_img.view(np.int8)).cuda()
    B = torch.as_tensor(b_img.view(np.int8)).cuda()
    D = torch.zeros(128 * N, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = L.umma_probe_run(A.data_ptr(), a_img.nbytes, B.data_ptr(), b_img.nbytes, N, a_mn, b_mn, *a_fields,
                          *b_fields, f8, D.data_ptr(), err.data_ptr())
    assert rc == 0 and err.item() == 0
    return D.cpu().numpy().reshape(128, N)


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_descriptor_fields(probe, a_mn, b_mn):
    rng = np.random.default_rng(a_mn * 2 + b_mn)
    M, N, K = 128, 128, 128
    A = rng.integers(-3, 4, size=(M, K)).astype(np.float32)
    B = rng.integers(-3, 4, size=(N, K)).astype(np.float32)
    ref = A @ B.T
    # K-major: image of A [M][K]; MN-major: image of A^T [K][M]
    a_img = canon_image(A.T if a_mn else A)
    b_img = canon_image(B.T if b_mn else B)
    kmaj = (128, K * 16, 256)                 # LBO, SBO, start step per 16-k MMA
    a_f = (M * 16, 128, 2 * M * 16) if a_mn else kmaj   # MN-major: LBO = K-group stride, SBO = MN-group stride
    b_f = (N * 16, 128, 2 * N * 16) if b_mn else kmaj
    D = run(probe, a_img, b_img, N, a_mn, b_mn, a_f, b_f)
    assert np.array_equal(D, ref)


def canon8_image(T):
    """Byte image of a [R][K] tile of E4M3 values in the 8-bit canonical K-major layout."""
    R, K = T.shape
    img = np.zeros(R * K, dtype=np.uint8)
    r, k = np.meshgrid(np.arange(R), np.arange(K), indexing="ij")
    off = (r >> 3) * (K * 8) + (k >> 4) * 128 + (r & 7) * 16 + (k & 15)
    bits = torch.as_tensor(T.astype(np.float32)).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    img[off.reshape(-1)] = bits.reshape(-1)
    return img


@pytest.mark.parametrize("N", [64, 128])
def test_e4m3_descriptor_fields(probe, N):
    """kind::f8f6f4 with E4M3 A and B: small integers (exact in E4M3 and in the FP32 sums)."""
    rng = np.random.default_rng(N)
    A = rng.integers(-4, 5, size=(128, 128)).astype(np.float32)
    B = rng.integers(-4, 5, size=(N, 128)).astype(np.float32)
    kmaj8 = (128, 128 * 8, 256)   # LBO, SBO = 8 K, start step per 32-k MMA
    D = run(probe, canon8_image(A), canon8_image(B), N, 0, 0, kmaj8, kmaj8, f8=1)
    assert np.array_equal(D, A @ B.T)
