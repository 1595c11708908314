"""Shared set-up of the GPU parity tests (inputs from synth, expected values from oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

ABC = (1.0, 1.0, 1.0, -1.0)
RHO = 1.5
# relative-L2 tolerances per application (FP64, FP32, FP16 storage); BF16 storage is
# reported against 2 x 2^-8 (one rounding of input, link and output at unit roundoff 2^-8);
# double-float (two FP32 words, about 2^-46 per operation) is held to the FP64 bound
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 1e-3, "bf16": 8e-3, "df64": 1e-12}


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()
