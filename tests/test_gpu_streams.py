"""Calls on two streams at once: each stream has its own library workspace, so
products that both need scratch memory (the emulation's slices, split-k
partials) run concurrently and still equal the same calls made one after the
other, bit for bit."""
import pytest

from gpu_util import device_operands, lib, out_tensor

pytestmark = pytest.mark.gpu


def test_two_streams_concurrent_products_equal_serial():
    import torch
    cosma = lib()
    jobs = [("f64_emu_bf16", (1024, 768, 2048)), ("f32", (96, 80, 6000)),
            ("bf16", (200, 136, 20000)), ("f32_emu_tf32", (256, 384, 3000))]
    ops = []
    for i, (dt, (m, n, k)) in enumerate(jobs):
        A, B = device_operands(m, n, k, dt, "uniform", 20 + i)
        Cs, _ = out_tensor(m, n, dt)
        Cc, _ = out_tensor(m, n, dt)
        ops.append((dt, A, B, Cs, Cc))
    # serial reference on the current stream
    for dt, A, B, Cs, _ in ops:
        cosma.gemm(A, B, Cs, dt)
    torch.cuda.synchronize()
    # the same calls spread over two streams, several rounds, no synchronisation between
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for s in streams:
        s.wait_stream(torch.cuda.current_stream())
    for _ in range(4):
        for i, (dt, A, B, _, Cc) in enumerate(ops):
            with torch.cuda.stream(streams[i % 2]):
                cosma.gemm(A, B, Cc, dt)
    torch.cuda.synchronize()
    assert cosma.cosma_stream_status(torch.cuda.current_stream().cuda_stream) == 0
    for dt, _, _, Cs, Cc in ops:
        assert torch.equal(Cs, Cc), dt
