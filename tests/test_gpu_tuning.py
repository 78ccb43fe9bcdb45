"""Launch knobs change launch shapes, never results: the CUDA path under
extreme knob values against the oracle (single images, including the graph
replayed after each change, and a batch)."""
import numpy as np
import pytest

from tests.test_gpu_parity import cells, gpu, oracle_cells

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# red_budget 1 sets nearly every residual column aside after one step of the
# wide pass and resumes it in the deep pass; 0 runs the deep pass alone
SETTINGS = [
    {"uf_items": 1, "uf_compact": 1, "red_warps": 1, "batch_threads": 0, "red_budget": 1},
    {"uf_items": 64, "uf_compact": 64, "red_warps": 16, "batch_threads": 1, "red_budget": 0},
    {"uf_items": 2, "uf_compact": 8, "red_warps": 4, "batch_threads": 3, "red_budget": 8},
    {"uf_items": 8, "uf_compact": 1, "red_warps": 16, "batch_threads": 2, "red_budget": 1024},
]


def test_knobs_do_not_change_results(cr, oracle_mod):
    from paper_2005_12692_gb300 import autotune as at
    from paper_2005_12692_gb300 import synth
    imgs = [synth.grf((257, 300), 4.0, 10), synth.salted(synth.grf((33, 40, 29), 3.0, 12), 0.01, 13)]
    exp = [oracle_cells(oracle_mod, im) for im in imgs]
    batch = [synth.grf(s, 2.0, 900 + i) for i, s in enumerate([(40, 33), (64, 64), (17, 90)])]
    single = [cells(gpu(cr, im)) for im in batch]
    vols = [synth.salted(synth.grf(s, 2.5, 950 + i), 0.02, 960 + i) for i, s in enumerate([(24, 30, 21), (31, 17, 26)])]
    vexp = [oracle_cells(oracle_mod, v) for v in vols]
    try:
        for s in SETTINGS:
            at.apply(s)
            for im, e in zip(imgs, exp):
                for _ in range(3):  # the third 2D call replays the graph captured under these knobs
                    assert cells(gpu(cr, im)) == e, s
            bp = cr.cr_persistence_batched([torch.from_numpy(b).cuda() for b in batch], keep_zero=True)
            for i in range(len(batch)):
                assert cells(bp.image(i).numpy()) == single[i], s
            bv = cr.cr_persistence_batched([torch.from_numpy(v).cuda() for v in vols], keep_zero=True)
            for i in range(len(vols)):
                assert cells(bv.image(i).numpy()) == vexp[i], s
    finally:
        at.apply(at.DEFAULTS)
