"""What the trained guidance network gains over the plain corner phase (needs
a GB300).

The network is trained by the library's own kernels on rows that the method
produces (plain corner phases of 12 seed-generated 2000 x 8000 power-law LPs)
and compared with the plain corner phase on held-out seeds.  The plain run
judges the network: a held column is wrong when the plain corner did not
leave it at the bound it was held at.  Asserted: the network learned (its loss
falls below the entropy of the label frequency), its holds are precise, and
with the fallback the guided result is never worse than the phase-1 point.
The time ratio is measured and printed, not asserted: on this LP family even
holding every column the plain corner leaves at its bound does not shorten
the corner phase, so the expected ratio is about 1.
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
G = pytest.importorskip("paper_2511_13894_gb300.guide")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _lp(seed):
    return lpgen.power_law_lp(2000, 8000, 100, lpgen.workload_seed(0, 7, seed), kmax=500, name="power_law_m2k_n8k")


def test_trained_network_against_the_plain_corner_phase():
    train_lps = [_lp(s) for s in range(12)]
    data = G.build_dataset(train_lps, [s + 1 for s in range(12)])
    assert data["rows"] > 10000
    pos = float(data["labels"][:data["rows"]].float().mean().item())
    net = P.Guide(seed=0)
    losses = G.train(net, data, steps=3000, batch=4096, lr=1e-3, seed=5)
    entropy = -(pos * np.log(pos) + (1 - pos) * np.log(1 - pos))
    assert float(np.mean(losses[-50:])) < 0.9 * entropy
    ratios = []
    for s in (1000, 1001):
        r = G.compare(net, _lp(s), s + 1, threshold=0.9, guided_max_iters=2 * 64 * 1024)
        print("held-out LP %d: plain %s %d it %.3f s | held %d of %d eligible, precision %.3f | guided %s %d it, "
              "fell back %s | time ratio plain/guided %.3f" % (
                  s, r["plain_status"], r["plain_iters"], r["plain_seconds"], r["held"], r["eligible"],
                  r["precision"] or 0.0, r["guided_status"], r["guided_iters"], r["fell_back"], r["speedup"]))
        assert r["held"] == r["held_host"] > 0
        assert r["precision"] >= 0.9
        if r["plain_status"] == "CORNER_DONE":
            assert r["final_status"] == "CORNER_DONE"
        assert r["final_corner_measure"] <= r["phase1_corner_measure"]
        assert r["final_rel_kkt"] <= max(1e-6, r["plain_rel_kkt"]) * (1 + 1e-9)
        ratios.append(r["speedup"])
    print("time-to-corner ratio plain/guided: %s" % ", ".join("%.3f" % v for v in ratios))
