"""cosma_gemm captured into a CUDA graph (every dtype): once the library's
workspace has been sized by an eager call, the whole path -- planning, operand
preparation, the main kernel (cooperative launches included), the Reduce -- is
recorded, and a replay on new input values equals an eager call on them bit for
bit (the computation does not depend on how it is launched)."""
import pytest

from gpu_util import device_operands, lib, out_tensor

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "f64_emu_bf16", "f32_emu_tf32"])
@pytest.mark.parametrize("shape", [(300, 260, 700), (96, 80, 6000)])
def test_gemm_graph_replay_equals_eager(dtype, shape):
    import torch
    import cosma_inputs as ci
    from cosma_inputs import device as cid
    from gpu_util import GEN_DT
    cosma = lib()
    m, n, k = shape
    A, B = device_operands(m, n, k, dtype, "uniform", 1)
    C, _ = out_tensor(m, n, dtype)
    cosma.gemm(A, B, C, dtype)  # sizes the workspace outside the capture
    torch.cuda.synchronize()
    Cg, _ = out_tensor(m, n, dtype)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cosma.gemm(A, B, Cg, dtype)
    # new values in the same buffers, then replay and an eager call
    cid.fill(A, "uniform", GEN_DT[dtype], 2, ci.STREAM_A)
    cid.fill(B, "uniform", GEN_DT[dtype], 2, ci.STREAM_B)
    graph.replay()
    cosma.gemm(A, B, C, dtype)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    assert torch.equal(Cg, C)


@pytest.mark.parametrize("dtype", ["f32_emu_tf32", "f64_emu_bf16"])
def test_graph_stays_valid_after_the_workspace_grows(dtype):
    """A later call that needs a larger workspace on the stream whose arena the
    capture recorded takes a new buffer; the recorded one is kept until
    cosma_finalize, so a replay still equals the eager call bit for bit."""
    import torch
    cosma = lib()
    m, n, k = 300, 260, 700
    A, B = device_operands(m, n, k, dtype, "uniform", 1)
    C, _ = out_tensor(m, n, dtype)
    side = torch.cuda.Stream()   # a new stream: a new, small arena
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cosma.gemm(A, B, C, dtype)
    torch.cuda.synchronize()
    Cg, _ = out_tensor(m, n, dtype)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cosma.gemm(A, B, Cg, dtype)
    # a product whose workspace is many times larger grows that arena
    A2, B2 = device_operands(2048, 2048, 4096, dtype, "uniform", 3)
    C2, _ = out_tensor(2048, 2048, dtype)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        cosma.gemm(A2, B2, C2, dtype)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    assert torch.equal(Cg, C)
