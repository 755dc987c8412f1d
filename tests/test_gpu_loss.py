"""GPU parity of snp_mse_loss (the differentiation workload's squared-error loss)
against the FP64 oracle: value, gradient, ragged and misaligned sizes, the empty
case, determinism and CUDA-graph capture."""
import numpy as np
import pytest
import torch

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2510_08491_gb300 import build
    build.build()
    from paper_2510_08491_gb300.render import Renderer
    return Renderer(0)


def _pair(n, seed, offset=0):
    g = torch.Generator("cuda").manual_seed(seed)
    a = torch.rand(n + offset, device="cuda", generator=g)[offset:]
    b = torch.rand(n + offset, device="cuda", generator=g)[offset:]
    return a, b


@pytest.mark.parametrize("n,offset", [(1, 0), (3, 0), (5, 1), (1023, 0), (3 * 7919, 1), (3 * 1280 * 720, 0)])
def test_loss_and_gradient_match_oracle(R, n, offset):
    img, tgt = _pair(n, n, offset)
    loss, dL = R.mse_loss(img, tgt)
    torch.cuda.synchronize()
    ref_loss, ref_g = O.mse_loss(img.cpu().numpy(), tgt.cpu().numpy())
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss + 1e-30
    err = np.abs(dL.cpu().numpy().astype(np.float64) - ref_g)
    assert (err <= 1e-6 * np.abs(ref_g) + 1e-30).all(), err.max()


def test_empty_and_deterministic(R):
    e = torch.empty(0, device="cuda")
    loss, _ = R.mse_loss(e, e)
    assert loss.item() == 0.0
    img, tgt = _pair(3 * 640 * 480, 7)
    l1, _ = R.mse_loss(img, tgt)
    l1 = l1.clone()
    l2, _ = R.mse_loss(img, tgt)
    assert torch.equal(l1, l2)


def test_graph_capture(R):
    img, tgt = _pair(3 * 320 * 240, 11)
    dL = torch.empty_like(img)
    loss = torch.empty(1, device="cuda")
    R.mse_loss(img, tgt, dL, loss)
    torch.cuda.synchronize()
    ref = loss.clone()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            R.mse_loss(img, tgt, dL, loss, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        loss.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(loss, ref)
