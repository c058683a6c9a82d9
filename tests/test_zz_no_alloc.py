"""pic_diag_noalloc: diagnostics for callers that must not allocate device memory.

Some callers cannot let the library allocate after set-up (a fixed device
memory budget handed over at creation, latency-critical loops where
cudaMalloc/cudaFree would synchronise the device, code running inside another
library's callbacks).  pic_diag_noalloc runs the same reductions as pic_diag
with its scratch in a fixed device array.  This test calls it through the
C-ABI and checks that two calls in a row give what pic_diag gives, for every
diagnostic kind, on both precisions, that the calls allocate nothing (the
handle's device memory comes from counting hooks, and pic_diag, called after,
is seen to allocate through them), and that an over-long request is refused.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_1204_0838_gb300 import pic, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12  # same kernels, different scratch: only atomic summation order differs


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    pic.lib()


class CountingMemory(pic.TorchMemory):
    """The torch-backed pic_alloc hooks, counting the allocations made."""

    def __init__(self):
        self.allocs = 0
        super().__init__()

    def _alloc(self, nbytes, ctx):
        self.allocs += 1
        return super()._alloc(nbytes, ctx)


def _sim(precision, memory=None):
    cfg = W.config("c1", crop=(96, 24, 24))
    cfg["x0"] = -48 * cfg["dx"]
    cfg["fwhm"], cfg["waist"], cfg["t_peak"] = 4e-15, 3e-6, 40 * cfg["dx"] / W.C0
    cfg["prof_x"], cfg["prof_n"] = [0.0, 2e-6, 1.0], [0.0, 0.02, 0.02]
    g = pic.Sim(cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dy"], cfg["dz"], cfg["lambda0"],
                x0=cfg["x0"], periodic_x=False, precision=precision, seed=cfg["seed"],
                window=cfg["window"], memory=memory)
    g.add_species(cfg["prof_x"], cfg["prof_n"], cfg["ppc"], loading=cfg["loading"])
    g.add_laser(cfg["a0"], cfg["waist"], cfg["fwhm"], cfg["lambda0"], cfg["x_focus"], cfg["t_peak"])
    g.step(40)
    return g, cfg


def _close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= TOL * scale


def _requests(nx):
    return [
        (pic.PIC_DIAG_EX_LINEOUT, nx, {}),
        (pic.PIC_DIAG_FIELD_ENERGY, 1, {}),
        (pic.PIC_DIAG_CHARGE, 1, {"gamma_min": 1.0001}),
        (pic.PIC_DIAG_CHARGE, 1, {"gamma_min": 0.0}),
        (pic.PIC_DIAG_SPECTRUM, 64, {"e_min": 0.0, "e_max": 0.2}),
    ]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_diag_allocates_nothing(precision):
    mem = CountingMemory()
    g, cfg = _sim(precision, memory=mem)
    before = mem.allocs
    assert before > 0  # the handle's own memory came through the hooks
    results = [pic.pic_diag_noalloc(g.h, kind, length, **kw) for kind, length, kw in _requests(cfg["nx"])]
    assert mem.allocs == before
    # the check is sensitive: pic_diag's first request allocates its scratch through the hooks
    ref = [pic.pic_diag(g.h, kind, length, **kw) for kind, length, kw in _requests(cfg["nx"])]
    assert mem.allocs > before
    for a, b in zip(results, ref):
        assert _close(a, b)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_diag_matches_pic_diag_on_two_calls(precision):
    g, cfg = _sim(precision)
    requests = _requests(cfg["nx"])
    for kind, length, kw in requests:
        ref = pic.pic_diag(g.h, kind, length, **kw)
        first = pic.pic_diag_noalloc(g.h, kind, length, **kw)
        second = pic.pic_diag_noalloc(g.h, kind, length, **kw)
        assert np.abs(ref).max() > 0
        assert _close(first, ref), (kind, first[:4], ref[:4])
        assert _close(second, ref), (kind, second[:4], ref[:4])
    g.step(1)  # the state moves on: the shared scratch must not carry old sums
    for kind, length, kw in requests:
        assert _close(pic.pic_diag_noalloc(g.h, kind, length, **kw), pic.pic_diag(g.h, kind, length, **kw))
    g.close()


def test_noalloc_diag_rejects_results_longer_than_its_scratch():
    g, _ = _sim("fp32")
    with pytest.raises(pic.PicError) as e:
        pic.pic_diag_noalloc(g.h, pic.PIC_DIAG_SPECTRUM, 65537, e_min=0.0, e_max=1.0)
    assert e.value.code == -1
    assert "PIC_NOALLOC_MAX_LEN" in str(e.value)
    out = pic.pic_diag_noalloc(g.h, pic.PIC_DIAG_SPECTRUM, 65536, e_min=0.0, e_max=1.0)
    assert out.size == 65536
    g.close()
