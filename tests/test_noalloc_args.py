"""The binding of the allocation-free scan checks every tensor before anything
reaches the device (the kernel trusts the sizes it is given, so a short buffer
would be read or written out of bounds rather than rejected).  Runs on the CPU:
each case fails on its own check before the device check, and tensors that are
not on a CUDA device are refused last."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def ebr():
    from paper_2511_22460_gb300 import _build
    _build.build()
    from paper_2511_22460_gb300 import ebr as mod
    return mod


def _args(n=1000, d=16, k=10):
    f32 = torch.float32
    return dict(emb=torch.zeros((n, d), dtype=f32), h_u=torch.zeros(d, dtype=f32),
                wide=torch.zeros(n, dtype=f32),
                filt=torch.zeros((n + 63) // 64, dtype=torch.int64), k=k,
                out_ids=torch.zeros(k, dtype=torch.int32), out_scores=torch.zeros(k, dtype=f32))


def _call(ebr, **a):
    ebr.scan_topk_noalloc(a["emb"], a["h_u"], a["wide"], a["filt"], a["k"], a["out_ids"],
                          a["out_scores"])


@pytest.mark.parametrize("change,match", [
    (dict(emb=torch.zeros((1000, 16), dtype=torch.bfloat16)), "float32"),
    (dict(emb=torch.zeros((16, 1000), dtype=torch.float32).t()), "contiguous"),
    (dict(emb=torch.zeros(16000, dtype=torch.float32)), "2-D"),
    (dict(emb=torch.zeros((1000, 12), dtype=torch.float32)), "d in"),
    (dict(k=0), "k must"),
    (dict(k=1025), "k must"),
    (dict(h_u=torch.zeros(15, dtype=torch.float32)), "h_u needs"),
    (dict(h_u=torch.zeros(16, dtype=torch.float64)), "h_u must have dtype"),
    (dict(wide=torch.zeros(999, dtype=torch.float32)), "wide needs"),
    (dict(filt=torch.zeros(15, dtype=torch.int64)), "filter needs"),
    (dict(filt=torch.zeros(16, dtype=torch.int32)), "filter must have dtype"),
    (dict(out_ids=torch.zeros(9, dtype=torch.int32)), "out_ids needs"),
    (dict(out_scores=torch.zeros(9, dtype=torch.float32)), "out_scores needs"),
    (dict(out_ids=torch.zeros(20, dtype=torch.int32)[::2]), "out_ids must be contiguous"),
    (dict(), "CUDA tensor"),  # every shape right: refused because it is not on a GPU
], ids=["bf16", "strided", "1d", "bad_d", "k0", "k_big", "short_h", "h_f64", "short_wide",
        "short_filter", "filter_i32", "short_ids", "short_scores", "strided_ids", "cpu"])
def test_rejected_before_launch(ebr, change, match):
    a = _args()
    a.update(change)
    with pytest.raises(ValueError, match=match):
        _call(ebr, **a)
