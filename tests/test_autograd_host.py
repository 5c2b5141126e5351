"""Host logic of the autograd wrapper, on the CPU with a stand-in for the
Rasterizer (no library call): gradients flow back to every parameter tensor,
and a backward after a newer forward through the same Rasterizer raises
instead of differentiating with the newer forward's lists."""
import pytest

torch = pytest.importorskip("torch")

from paper_2603_09277_gb300.rasterize import PARAM_KEYS, rasterize  # noqa: E402


class StandIn:
    """Records calls; its 'backward' returns each parameter's values as the
    gradient so that the flow can be checked."""

    def __init__(self, n=4, pixels=6):
        self.image = torch.zeros(pixels, 3)
        self.entropy = torch.zeros(pixels)
        self.forward_count = 0
        self.calls = []

    def preprocess(self, p):
        self.calls.append("preprocess")
        self.p = p

    def bin_sort(self):
        self.calls.append("bin_sort")

    def render_fwd(self):
        self.calls.append("render_fwd")
        self.image.fill_(float(self.forward_count + 1))

    def render_bwd(self, p, g_image, g_entropy):
        self.calls.append("render_bwd")
        return {k: p[k].detach() * 2.0 for k in PARAM_KEYS}


def _params(n=4):
    g = torch.Generator().manual_seed(0)
    shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity_logits": (n,),
              "sh": (n, 16, 3)}
    return {k: torch.randn(*s, generator=g).requires_grad_(True) for k, s in shapes.items()}


def test_gradients_reach_every_parameter():
    r = StandIn()
    p = _params()
    img, ent = rasterize(p, r)
    (img.sum() + ent.sum()).backward()
    assert r.calls == ["preprocess", "bin_sort", "render_fwd", "render_bwd"]
    for k in PARAM_KEYS:
        assert torch.equal(p[k].grad, p[k].detach() * 2.0), k


def test_backward_after_a_newer_forward_raises():
    r = StandIn()
    p = _params()
    img1, _ = rasterize(p, r)
    img2, _ = rasterize(p, r)
    with pytest.raises(RuntimeError, match="another forward"):
        img1.sum().backward()
    img2.sum().backward()  # the latest forward still differentiates
    assert torch.equal(p["means"].grad, p["means"].detach() * 2.0)
