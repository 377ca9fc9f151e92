"""Learned corner guidance: the CUDA path vs the CPU oracle (needs a GB300).

* features (restart history, column norms, corner objective, RMS scaling)
  within one BF16 rounding of the FP64 oracle; eligibility equal;
* the BF16 network: probabilities within 1e-2 of the FP64 MLP on the same
  (BF16-representable) weights and inputs; the minibatch gradient within
  2e-2 relative per tensor of the FP64 gradient (BF16 activations and
  gradients in the weight products, FP32 accumulation); one Adam step equal
  to the oracle's where the gradient's sign is unambiguous;
* the guided corner phase with a given hold mask, and with the network's
  hold decisions, at the corner-phase parity bar (equal iteration counts,
  x within 1e-7); the fallback decision equal to the oracle's;
* the training rows: eligible columns in order, labels equal to the oracle's.
"""
import numpy as np
import pytest

import lpgen
import oracle
from oracle import guide as oguide
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2511_13894_gb300.pdhgc")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BF16_REL = 2.0 ** -7  # one BF16 unit in the last place, relative


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def to_bf16_bits(x):
    """Round-to-nearest-even FP32 -> BF16 bit patterns (uint16)."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) >> 16).astype(np.uint16)


def bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_round(x):
    return bf16_value(to_bf16_bits(x)).reshape(np.shape(x))


def feat_tensor(F):
    """n x 18 values -> CUDA n x 32 bfloat16 (zero padded), and the exact values."""
    bits = np.zeros((F.shape[0], 32), dtype=np.uint16)
    bits[:, :18] = to_bf16_bits(F).reshape(F.shape)
    t = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).cuda()
    return t, bf16_value(bits[:, :18])


def feat_values(t):
    bits = t.view(torch.int16).cpu().numpy().view(np.uint16)
    return bf16_value(bits)


def rounded_weights(seed, b3=0.3):
    """Oracle-layout weights whose matrices are exactly BF16 (the kernels'
    operands) and whose biases are FP32 values."""
    w = omlp.init_weights(seed)
    rng = np.random.default_rng(seed + 50)
    w["b1"] = rng.standard_normal(64) * 0.1
    w["b2"] = rng.standard_normal(64) * 0.1
    w["b3"] = np.asarray(b3)
    for k in ("W1", "W2", "w3"):
        w[k] = bf16_round(w[k])
    for k in ("b1", "b2", "b3"):
        w[k] = np.asarray(w[k], dtype=np.float32).astype(np.float64)
    return w


def pack(w):
    return np.concatenate([w["W1"].ravel(), w["b1"], w["W2"].ravel(), w["b2"], w["w3"],
                           np.atleast_1d(w["b3"])]).astype(np.float32)


def unpack(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for k, shape in (("W1", (64, 18)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,)),
                     ("b3", ())):
        size = int(np.prod(shape)) if shape else 1
        out[k] = v[o:o + size].reshape(shape) if shape else np.asarray(v[o])
        o += size
    return out


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------

FEATURE_CASES = {
    "bounded_ineq": lambda: lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(5), 5),
    "power_law": lambda: lpgen.power_law_lp(600, 2400, 60, seed=9, kmax=300),
}


@pytest.mark.parametrize("name", list(FEATURE_CASES))
def test_features_match_oracle(name):
    lp = FEATURE_CASES[name]()
    r1 = oracle.solve(lp)
    g = P.lp_from_dict(lp)
    rep = g.solve()
    assert rep["iters"] == r1["iters"] and rep["restarts"] == r1["restarts"]
    cp = dict(obj_seed=7)
    feat, elig = g.guide_features(obj_seed=7)
    F, E = oguide.features(r1, cp)
    got = feat_values(feat)
    assert np.all(got[:, 18:] == 0.0)
    got = got[:, :18]
    err = np.abs(got - F)
    assert np.all(err <= BF16_REL * np.abs(F) + 1e-30), float(np.max(err / (np.abs(F) + 1e-30)))
    assert np.array_equal(elig.cpu().numpy().astype(bool), E)


# --------------------------------------------------------------------------
# network: forward, gradient, Adam, training
# --------------------------------------------------------------------------

def _random_inputs(n, seed):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((n, 18))
    y = (rng.random(n) < 0.35).astype(np.uint8)
    return F, y


def test_forward_matches_oracle_mlp():
    F, _ = _random_inputs(3000, 1)  # 187.5 tiles of 16: a ragged last tile
    feat, X = feat_tensor(F)
    w = rounded_weights(3)
    g = P.Guide(seed=0)
    g.set_weights(pack(w))
    p = g.infer(feat).cpu().numpy().astype(np.float64)
    ref, _ = omlp.forward(w, X)
    assert np.max(np.abs(p - ref)) <= 1e-2
    assert np.mean(np.abs(p - ref)) <= 2e-3


@pytest.mark.parametrize("batch", [1000, 64])
def test_gradient_matches_oracle(batch):
    F, y = _random_inputs(5000, 2)
    feat, X = feat_tensor(F)
    lab = torch.from_numpy(y).cuda()
    w = rounded_weights(4)
    g = P.Guide(seed=0)
    g.set_weights(pack(w))
    idx = np.random.default_rng(5).integers(0, 5000, size=batch).astype(np.int32)
    grad, loss = g.grad(feat, lab, idx)
    ref = omlp.gradients(w, X[idx], y[idx].astype(np.float64))
    got = unpack(grad)
    for k in ref:
        a, b = np.atleast_1d(got[k]), np.atleast_1d(ref[k])
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= 2e-2, (k, rel)
    ref_loss = omlp.loss_of(w, X[idx], y[idx].astype(np.float64))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    # no update: the weights are unchanged
    assert np.array_equal(g.get_weights(), pack(w))


def test_one_adam_step_matches_oracle():
    F, y = _random_inputs(4000, 3)
    feat, X = feat_tensor(F)
    lab = torch.from_numpy(y).cuda()
    w = rounded_weights(6)
    g = P.Guide(seed=0)
    g.set_weights(pack(w))
    batch, seed, lr = 512, 77, 1e-3
    losses = g.train(feat, lab, rows=4000, batch=batch, steps=1, lr=lr, seed=seed)
    # the minibatch rows: SplitMix64(seed, s) mod rows for s < batch (step 0)
    idx = (oracle.splitmix64(seed, batch) % np.uint64(4000)).astype(np.int64)
    ref_g = omlp.gradients(w, X[idx], y[idx].astype(np.float64))
    assert abs(losses[0] - omlp.loss_of(w, X[idx], y[idx].astype(np.float64))) <= 1e-3 * losses[0]
    w_ref = omlp.adam_step({k: np.array(v, dtype=np.float64, copy=True) for k, v in w.items()}, ref_g, {}, lr=lr)
    got = unpack(g.get_weights())
    for k in w:
        gk = np.atleast_1d(ref_g[k])
        big = np.abs(gk) >= 0.05 * np.max(np.abs(gk))
        d_got = np.atleast_1d(got[k] - w[k])
        d_ref = np.atleast_1d(w_ref[k] - w[k])
        assert np.all(np.abs(d_got[big] - d_ref[big]) <= 1e-2 * lr), k
        # every step has Adam's first-step size: lr * |g| / (|g| + eps)
        assert np.all(np.abs(d_got) <= lr * (1 + 1e-3)), k


def test_training_reduces_the_loss():
    F, _ = _random_inputs(20000, 4)
    y = ((F[:, 0] + 0.5 * F[:, 3] - F[:, 11]) > 0.3).astype(np.uint8)
    feat, _ = feat_tensor(F)
    lab = torch.from_numpy(y).cuda()
    g = P.Guide(seed=1)
    losses = g.train(feat, lab, rows=20000, batch=1024, steps=400, lr=3e-3, seed=9)
    assert np.all(np.isfinite(losses))
    assert float(np.mean(losses[-20:])) < 0.5 * float(np.mean(losses[:5]))
    p = g.infer(feat).cpu().numpy()
    acc = float(np.mean((p >= 0.5) == (y == 1)))
    assert acc >= 0.95


# --------------------------------------------------------------------------
# guided corner phase
# --------------------------------------------------------------------------

def _hold_near_bound(r1, cp, count):
    model = r1["model"]
    elig = oguide.eligible(r1, dict(oracle.CORNER_DEFAULTS, **cp))
    x1 = model.Dc * r1["x_hat"]
    dist = np.where(elig, np.minimum(x1 - model.l, model.u - x1), np.inf)
    hold = np.zeros(model.n, dtype=bool)
    hold[np.argsort(dist, kind="stable")[:count]] = True
    return hold


@pytest.mark.parametrize("device_mask", [False, True])
def test_guided_corner_with_mask_matches_oracle(device_mask):
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(9), 9)
    r1 = oracle.solve(lp)
    cp = dict(obj_seed=4)
    hold = _hold_near_bound(r1, cp, 12)
    ref = oracle.corner_phase(r1, cp, hold=hold)
    g = P.lp_from_dict(lp)
    g.solve()
    mask = torch.from_numpy(hold.astype(np.uint8)).cuda() if device_mask else hold
    rep, grep = g.corner_phase_guided(hold=mask, fallback=False, obj_seed=4)
    assert grep["held"] == ref["info"]["held"] == 12
    assert grep["eligible"] == int(oguide.eligible(r1, dict(oracle.CORNER_DEFAULTS, **cp)).sum())
    assert rep["status"] == ref["status"] and rep["iters"] == ref["iters"]
    assert rep["restarts"] == ref["restarts"]
    x, _, _ = g.get_solution(P.CORNER)
    xo, _, _ = oracle.unscale(r1["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(x, xo) <= 1e-7
    orep = oracle.kkt_report(r1["model"], ref["x_hat"], ref["y_hat"])
    for k in ("off_bound_p", "candidates", "corner_measure"):
        assert rep[k] == orep[k], k


def test_guided_fallback_matches_oracle():
    lp = lpgen.small_face_lp(10)
    r1 = oracle.solve(lp)
    cp = dict(obj_seed=1, max_iters=4096)
    hold = lp["x_star"] > 0
    ref = oguide.guided_corner_phase(r1, hold, cp)
    assert ref["fell_back"]
    g = P.lp_from_dict(lp)
    g.solve()
    rep, grep = g.corner_phase_guided(hold=hold, fallback=True, obj_seed=1, max_iters=4096)
    assert grep["fell_back"] == 1 and grep["status_name"] == "GUIDE_FALLBACK"
    assert grep["guided_iters"] == ref["guided"]["iters"]
    plain = g.corner_phase(obj_seed=1, max_iters=4096)
    assert rep["iters"] == plain["iters"] == ref["result"]["iters"]
    x_fb, _, _ = g.get_solution(P.CORNER)
    xo, _, _ = oracle.unscale(r1["model"], ref["result"]["x_hat"], ref["result"]["y_hat"])
    assert rel_err(x_fb, xo) <= 1e-7


def test_guided_corner_with_network_matches_oracle():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(11), 11)
    r1 = oracle.solve(lp)
    cp = dict(obj_seed=5)
    w = rounded_weights(8, b3=1.0)
    w["w3"] = 4.0 * w["w3"]  # spread the logits (still exactly BF16)
    net = P.Guide(seed=0)
    net.set_weights(pack(w))
    g = P.lp_from_dict(lp)
    g.solve()
    feat, elig = g.guide_features(obj_seed=5)
    p_gpu = net.infer(feat).cpu().numpy().astype(np.float64)
    p_ref, E = oguide.predict(w, r1, cp)
    err = float(np.max(np.abs(p_gpu - p_ref)))
    assert err <= 1e-2
    # a threshold in the widest gap of the eligible probabilities that leaves
    # at least 5 columns on each side; the gap is wider than twice the error,
    # so that both sides take the same hold decisions
    pe = np.sort(p_ref[E])
    gaps = np.diff(pe[4:len(pe) - 4])
    k = 4 + int(np.argmax(gaps))
    assert pe[k + 1] - pe[k] > 2 * err
    thr = 0.5 * (pe[k] + pe[k + 1])
    hold = oguide.hold_mask(p_ref, E, thr)
    assert np.array_equal(hold, (p_gpu >= thr) & elig.cpu().numpy().astype(bool))
    ref = oracle.corner_phase(r1, cp, hold=hold)
    rep, grep = g.corner_phase_guided(guide=net, threshold=thr, fallback=False, obj_seed=5)
    assert grep["held"] == ref["info"]["held"] == int(hold.sum()) > 0
    assert rep["status"] == ref["status"] and rep["iters"] == ref["iters"]
    x, _, _ = g.get_solution(P.CORNER)
    xo, _, _ = oracle.unscale(r1["model"], ref["x_hat"], ref["y_hat"])
    assert rel_err(x, xo) <= 1e-7


def test_dataset_rows_and_labels():
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(12), 12)
    r1 = oracle.solve(lp)
    rc = oracle.corner_phase(r1, dict(obj_seed=3))
    g = P.lp_from_dict(lp)
    g.solve()
    g.corner_phase(obj_seed=3)
    feat_all, elig = g.guide_features(obj_seed=3)
    E = elig.cpu().numpy().astype(bool)
    cap = int(E.sum()) + 5
    fbuf = torch.zeros((cap, 32), dtype=torch.bfloat16, device="cuda")
    lbuf = torch.full((cap,), 7, dtype=torch.uint8, device="cuda")
    count = g.dataset_append(fbuf, lbuf, 2)
    assert count == 2 + int(E.sum())
    rows = fbuf[2:count].view(torch.int16).cpu().numpy()
    assert np.array_equal(rows, feat_all.view(torch.int16).cpu().numpy()[E])
    lab = oguide.labels(r1["model"], rc["x_hat"], r1["x_hat"])
    assert np.array_equal(lbuf[2:count].cpu().numpy().astype(bool), lab[E])
    assert int(lbuf[count:].cpu().numpy().max()) == 7  # nothing written past the rows
    # too small a buffer: BUFFER, nothing written, count unchanged
    small = torch.zeros((3, 32), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(P.PdhgcError) as e:
        g.dataset_append(small, torch.zeros(3, dtype=torch.uint8, device="cuda"), 0)
    assert e.value.code == -11


def test_guided_corner_in_fp32_bulk_holds_exactly():
    # FP32-bulk phase 1 and a held corner phase: held columns end exactly at
    # their bound and the Section 3.1 rule is met
    lp = lpgen.with_bounds_and_inequalities(lpgen.small_face_lp(9), 9)
    g = P.lp_from_dict(lp)
    g.solve(precision=P.FP32_BULK)
    _, elig = g.guide_features(obj_seed=4)
    E = elig.cpu().numpy().astype(bool)
    x1, _, _ = g.get_solution(P.PHASE1)
    lb, ub = lp["lb"], lp["ub"]
    dl = np.where(np.isfinite(lb), x1 - lb, np.inf)
    du = np.where(np.isfinite(ub), ub - x1, np.inf)
    nb = np.where(dl <= du, lb, ub)
    hold = np.zeros(lp["n"], dtype=bool)
    hold[np.argsort(np.where(E, np.minimum(dl, du), np.inf), kind="stable")[:12]] = True
    rep, grep = g.corner_phase_guided(hold=hold, fallback=False, obj_seed=4)
    assert grep["held"] == 12
    assert rep["status_name"] == "CORNER_DONE" and rep["rel_p"] <= 1e-6 * (1 + 1e-9)
    x, _, _ = g.get_solution(P.CORNER)
    assert np.max(np.abs(x[hold] - nb[hold])) <= 1e-12 * (1 + np.max(np.abs(nb[hold])))


def test_tensor_core_wait_that_gives_up_reports_device_error():
    # failure detection without a fault: the completion waits of the tcgen05
    # inference kernel give up at once, the call returns DEVICE, and the
    # context stays usable
    F, _ = _random_inputs(1000, 7)
    feat, _ = feat_tensor(F)
    g = P.Guide(seed=0)
    g.set_weights(pack(rounded_weights(2)))
    p_ok = g.infer(feat).cpu().numpy()
    g.set_wait_limit(0)
    with pytest.raises(P.PdhgcError) as e:
        g.infer(feat)
    assert e.value.code == -10
    g.set_wait_limit(1 << 24)
    assert np.array_equal(g.infer(feat).cpu().numpy(), p_ok)
    assert float(torch.ones(4, device="cuda").sum().item()) == 4.0


def test_empty_hold_is_the_plain_corner_phase():
    lp = lpgen.small_face_lp(13)
    g = P.lp_from_dict(lp)
    g.solve()
    plain = g.corner_phase(obj_seed=6)
    x_plain, _, _ = g.get_solution(P.CORNER)
    rep, grep = g.corner_phase_guided(hold=np.zeros(lp["n"], dtype=bool), fallback=False, obj_seed=6)
    assert grep["held"] == 0 and rep["iters"] == plain["iters"]
    x, _, _ = g.get_solution(P.CORNER)
    assert np.array_equal(x, x_plain)


def test_free_columns_are_never_eligible():
    # columns of S made free (l = -inf, u = +inf) keep the constructed optimum
    # (their reduced cost is 0) and must not be offered for holding
    lp = lpgen.small_face_lp(14)
    free = np.nonzero(lp["x_star"] > 0)[0][:6]
    lp["lb"] = lp["lb"].copy()
    lp["lb"][free] = -np.inf
    r1 = oracle.solve(lp)
    g = P.lp_from_dict(lp)
    rep = g.solve()
    assert rep["iters"] == r1["iters"]
    feat, elig = g.guide_features(obj_seed=2)
    F, E = oguide.features(r1, dict(obj_seed=2))
    got = feat_values(feat)[:, :18]
    assert np.all(np.abs(got - F) <= BF16_REL * np.abs(F) + 1e-30)
    assert np.array_equal(elig.cpu().numpy().astype(bool), E)
    assert not E[free].any()


def test_weights_survive_save_and_load(tmp_path):
    # a file written by pdhgc_guide_save restores the same parameters (and the
    # same probabilities) in another network; a damaged or foreign file is
    # refused with IO and leaves the network unchanged
    w = rounded_weights(4)
    a = P.Guide(seed=0)
    a.set_weights(pack(w))
    path = tmp_path / "net.pdhgcgw"
    a.save(str(path))
    b = P.Guide(seed=7)
    before = b.get_weights()
    b.load(str(path))
    assert np.array_equal(b.get_weights(), a.get_weights())
    F, _ = _random_inputs(500, 2)
    feat, _ = feat_tensor(F)
    assert torch.equal(a.infer(feat), b.infer(feat))
    raw = bytearray(path.read_bytes())
    assert raw[:8] == b"PDHGCGW1" and len(raw) == 16 + 4 * P.GUIDE_PARAMS + 8
    raw[100] ^= 0x01
    bad = tmp_path / "bad.pdhgcgw"
    bad.write_bytes(bytes(raw))
    c = P.Guide(seed=7)
    with pytest.raises(RuntimeError, match="IO"):
        c.load(str(bad))
    with pytest.raises(RuntimeError, match="IO"):
        c.load(str(tmp_path / "missing.pdhgcgw"))
    assert np.array_equal(c.get_weights(), before)
