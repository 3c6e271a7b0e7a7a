"""The tcgen05 dense layer against the definition relu(A B^T + bias) in fp64,
rounded to bf16: agreement within one bf16 rounding (2^-8 relative) plus the
FP32 accumulation error."""
import numpy as np
import pytest
import torch

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2506_22609_b300 import build

    build.build()
    from paper_2506_22609_b300 import ludax

    ludax.lib()
    return ludax


def bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16)


# the last shape is the one bench.py times (every element checked)
@pytest.mark.parametrize("Mr,N,K", [(128, 256, 64), (256, 512, 256), (384, 512, 512), (2048, 512, 128),
                                    (16384, 512, 512), (65536, 512, 512)])
def test_dense_relu_matches_fp64(L, Mr, N, K):
    rng = np.random.default_rng(Mr + N + K)
    a = bf16(rng.normal(0, 1, (Mr, K)))
    b = bf16(rng.normal(0, 1 / np.sqrt(K), (N, K)))
    bias = torch.from_numpy(rng.normal(0, 0.1, N).astype(np.float32))
    out = torch.full((Mr, N), -1, dtype=torch.int16, device="cuda")
    L.ludax_dense_bf16_relu(a.view(torch.int16).cuda(), b.view(torch.int16).cuda(), bias.cuda(), out)
    torch.cuda.synchronize()
    assert L.ludax_device_error() == 0
    got = out.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    z = a.double().numpy() @ b.double().numpy().T + bias.double().numpy()
    ref = np.maximum(z, 0.0)
    tol = np.abs(ref) * 2.0 ** -8 + 1e-4 * np.sqrt(K)
    assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
    assert (got[z < -1e-3] == 0).all()  # clearly negative pre-activations are cut by the ReLU


def test_dense_relu_rejects_unsupported_shapes(L):
    a = torch.zeros(100, 64, dtype=torch.int16, device="cuda")
    b = torch.zeros(256, 64, dtype=torch.int16, device="cuda")
    out = torch.zeros(100, 256, dtype=torch.int16, device="cuda")
    with pytest.raises(L.LudaxError) as ei:
        L.ludax_dense_bf16_relu(a, b, torch.zeros(256, device="cuda"), out)
    assert ei.value.status == -3


@pytest.mark.parametrize("kind", ["lop3", "iadd", "shf", "imad", "imad_hi", "lop3_imad"])
def test_int_peak_microbenchmark_runs(L, kind):
    """The integer-issue microbenchmark counts its ops exactly and finishes."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ops = L.ludax_int_peak(kind, 64)
    torch.cuda.synchronize()
    assert ops == sms * 8 * 256 * 8 * 64
    with pytest.raises(L.LudaxError):
        L.ludax_int_peak(kind, 0)


def test_bounded_wait_expires_and_reports(L):
    """A device wait that nothing completes gives up after its limit, the
    expiry reaches the host as LUDAX_ERR_TIMEOUT through the error word, the
    word is cleared by reading it, and the context keeps working."""
    assert L.ludax_device_error() == 0
    L.ludax_selftest_wait(2_000_000)  # about a millisecond of clock
    torch.cuda.synchronize()
    assert L.ludax_device_error() == 2
    assert L.ludax_device_error() == 0
    a = torch.ones(128, 64, dtype=torch.bfloat16, device="cuda")
    b = torch.ones(256, 64, dtype=torch.bfloat16, device="cuda")
    out = torch.empty(128, 256, dtype=torch.int16, device="cuda")
    L.ludax_dense_bf16_relu(a.view(torch.int16), b.view(torch.int16), torch.zeros(256, device="cuda"), out)
    torch.cuda.synchronize()
    assert (out.view(torch.bfloat16).float() == 64.0).all()
    assert L.ludax_device_error() == 0
    with pytest.raises(L.LudaxError):
        L.ludax_selftest_wait(0)
