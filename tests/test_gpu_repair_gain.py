"""What the trained repair network gains over the method without it.

The network is trained on the GPU by the library's own kernels on pairs the
method generates from seeded object scenes (500k surfels, 1600x1200), then
evaluated on two held-out scene seeds and poses. The gain is a smaller
re-rendered area: tiles whose gate passes take the network's fill and leave
the ROI re-render (on these workloads 4-21% of the plain method's re-rendered
pixels at tau = 0.5). The cost is
bounded: the PSNR of the affiliated eye against the full render may drop by at
most 0.5 dB.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_30741_gb300 import build
    build.build()
    from paper_2609_30741_gb300 import repair_train as T
    dev = torch.device("cuda", 0)
    ctx, pairs = T.build_pairs("object", 4, 6, 7000, dev)
    w, hist, secs = T.train(ctx, pairs, 1500, 512, 1e-3, 7000, gate_weight=1.0)
    ev = T.evaluate(ctx, "object", [9100, 9101], 3, 123, 0.5, dev)
    return dict(w=w, hist=hist, ev=ev)


def test_training_lowers_the_loss(trained):
    h = trained["hist"]
    assert h[-1][1] < 0.7 * h[0][1], h


def test_gate_cuts_the_rerendered_area_at_bounded_cost(trained):
    ev = trained["ev"]
    print({k: round(v, 4) for k, v in ev.items()})
    assert ev["net_pixels"] > 0.0                         # holes filled by the network
    assert ev["roi_learned"] <= 0.98 * ev["roi_plain"]    # fewer re-rendered pixels
    assert ev["psnr_learned"] >= ev["psnr_plain"] - 0.5   # at most 0.5 dB lost
    assert ev["psnr_learned"] > ev["psnr_interp"]         # and far better than no re-render
