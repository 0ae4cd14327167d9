"""GPU parity of the learned scheduler (features, MLP inference, training).

Features: every one of the 12 values equals the oracle's (integer pieces are
exact; the log2 of a float64 quantity rounded to float32 agrees to 1e-5).
Inference: logits agree with the fp64 oracle forward to 1e-4 relative, and
the chosen class equals the oracle's argmax wherever the top two logits are
more than 1e-3 apart.  Training: one Adam step equals the oracle's step.
CC_ORDER_AUTO: whatever schedule is chosen, labels equal the union-find
labels.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from oracle import sched as so

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    import paper_2311_02811_gb300 as lib
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return lib


GRAPHS = {
    "rmat12": lambda: (1 << 12, *gg.rmat(12, seed=1)),
    "rmat16-sampled": lambda: (1 << 16, *gg.rmat(16, seed=2)),
    "grid60": lambda: (60 * 70, *gg.grid(60, 70, seed=3)),
    "path": lambda: (5000, *gg.path(5000, seed=4)),
    "er": lambda: (3000, *gg.er(3000, 9000, seed=5)),
    "caterpillar": lambda: (100 * 16, *gg.caterpillar(100, seed=6)),
    "components64": lambda: gg.components64(),
    "edgeless": lambda: (10, torch.empty(0, dtype=torch.int32), torch.empty(0, dtype=torch.int32)),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_graph_features_match_oracle(cc, name):
    n, s, d = GRAPHS[name]()
    want = so.features(n, s.numpy(), d.numpy())
    sg, dg = s.cuda(), d.cuda()
    g = cc.cc_init(n, sg, dg)
    got = cc.cc_graph_features(g)
    got2 = cc.cc_graph_features(g)  # the scratch is left clean: same answer again
    cc.cc_free(g)
    assert np.allclose(got, want, rtol=0, atol=1e-5), (got, want)
    assert np.array_equal(got, got2)


def test_batch_features_match_oracle(cc):
    vo, eo, s, d, _ = gg.batch_mix(24, seed=9, device="cuda", n_lo=200, n_hi=1e5)
    b = cc.cc_batch_init(vo, eo, s, d)
    got = cc.cc_batch_features(b)
    cc.cc_batch_free(b)
    sh, dh = s.cpu().numpy(), d.cpu().numpy()
    for g in range(24):
        a, e = int(eo[g]), int(eo[g + 1])
        want = so.features(int(vo[g + 1] - vo[g]), sh[a:e], dh[a:e])
        assert np.allclose(got[g], want, atol=1e-5), g


def _random_blob(rng):
    layers = []
    for ni, no in zip(so.LAYER_IN, so.LAYER_OUT):
        layers.append((rng.normal(scale=1.0 / np.sqrt(ni), size=(no, ni)), rng.normal(scale=0.1, size=no)))
    mean = rng.normal(size=12)
    std = rng.uniform(0.5, 2.0, 12)
    import struct
    out = b"CCMLP01\x00" + struct.pack("<4i", 12, 64, 3, 18)
    out += np.asarray(mean, np.float32).tobytes() + np.asarray(std, np.float32).tobytes()
    for w, b in layers:
        w32 = np.asarray(w, np.float32)
        # round to nearest even into the top 16 bits
        u = w32.view(np.uint32).astype(np.uint64)
        r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
        out += r.tobytes() + np.asarray(b, np.float32).tobytes()
    return out


def test_predict_matches_oracle_forward(cc):
    rng = np.random.default_rng(11)
    blob = _random_blob(rng)
    assert len(blob) == cc.cc_sched_blob_bytes()
    cc.cc_sched_load(blob)
    try:
        x = rng.normal(loc=5, scale=3, size=(300, 12)).astype(np.float32)
        cls, logits = cc.cc_sched_predict(x)
    finally:
        cc.cc_sched_load(None)
    mean, std, layers = so.parse_blob(blob)
    xs = (x.astype(np.float64) - mean.astype(np.float32)) * (1.0 / std.astype(np.float32)).astype(np.float32)
    want = so.mlp_forward(xs, layers)
    assert np.allclose(logits, want, rtol=1e-4, atol=1e-4)
    top2 = np.sort(want, axis=1)[:, -2:]
    clear = top2[:, 1] - top2[:, 0] > 1e-3
    assert (cls[clear] == np.argmax(want, axis=1)[clear]).all()


def test_train_step_matches_oracle(cc):
    rng = np.random.default_rng(12)
    P = cc.cc_sched_param_count()
    assert P == sum(i * o + o for i, o in zip(so.LAYER_IN, so.LAYER_OUT))
    p0 = rng.normal(scale=0.2, size=P).astype(np.float32)
    x = rng.normal(size=(64, 12)).astype(np.float32)
    y = rng.integers(0, 18, 64).astype(np.int32)
    lr = 1e-3
    p1, loss = cc.cc_sched_train_step(x, y, p0, lr)
    want_loss, g = so.loss_and_grad(p0.astype(np.float64), x.astype(np.float64), y)
    want = so.adam_step(p0.astype(np.float64), g, lr)
    assert abs(loss - want_loss) < 1e-4
    big = np.abs(g) > 1e-4
    assert np.allclose(p1[big], want[big], rtol=0, atol=lr * 1e-3 + 1e-6)
    assert (np.abs(p1 - p0) <= lr * 1.0001 + 1e-7).all()


def test_training_fits_a_learnable_rule(cc):
    """Labels that are a simple function of two features are learned."""
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 10, size=(2048, 12)).astype(np.float32)
    y = (np.where(x[:, 0] > 5, 17, 1) - np.where(x[:, 1] > 5, 1, 0)).astype(np.int32)
    blob, loss = cc.cc_sched_train(x, y, epochs=40, batch=128, lr=3e-3, seed=5)
    cc.cc_sched_load(blob)
    try:
        cls, _ = cc.cc_sched_predict(x)
    finally:
        cc.cc_sched_load(None)
    assert (cls == y).mean() > 0.95, (cls == y).mean()
    assert loss < 0.3


def test_auto_schedule_returns_exact_labels(cc):
    rng = np.random.default_rng(14)
    cc.cc_sched_load(_random_blob(rng))
    try:
        for name in ("rmat12", "grid60", "path", "components64"):
            n, s, d = GRAPHS[name]()
            want = oracle.uf_labels(n, s, d)
            sg, dg = s.cuda(), d.cuda()
            g = cc.cc_init(n, sg, dg)
            out = torch.empty(n, dtype=torch.int32, device="cuda")
            st = cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
            cc.cc_free(g)
            assert (out.cpu().numpy() == want).all()
            assert st.order in (2, 4, 0) and st.check_interval in (1, 2, 4)
        vo, eo, s, d, _ = gg.batch_mix(16, seed=15, device="cuda", n_lo=200, n_hi=5e4)
        b = cc.cc_batch_init(vo, eo, s, d)
        out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
        cc.cc_batch_run(b, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        cc.cc_batch_free(b)
        sh, dh, lab = s.cpu().numpy(), d.cpu().numpy(), out.cpu().numpy()
        for gi in range(16):
            a, e = int(eo[gi]), int(eo[gi + 1])
            want = oracle.uf_labels(int(vo[gi + 1] - vo[gi]), sh[a:e], dh[a:e])
            assert np.array_equal(lab[vo[gi]:vo[gi + 1]], want)
    finally:
        cc.cc_sched_load(None)
    # without weights AUTO is the plain order-2 synchronous schedule
    n, s, d = GRAPHS["grid60"]()
    sg, dg = s.cuda(), d.cuda()
    g = cc.cc_init(n, sg, dg)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st = cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
    cc.cc_free(g)
    assert (st.order, st.mode, st.check_interval) == (2, cc.CC_SYNC, 1)
    _, it, _, _ = oracle.contour_sync(n, s, d, 2)
    assert st.sweeps == it


def _constant_blob(cls):
    """A weight blob whose output is the one-hot bias of class cls whatever
    the features (every weight zero)."""
    rng = np.random.default_rng(0)
    blob = bytearray(_random_blob(rng))
    import struct
    hdr = 8 + 16 + 2 * 4 * 12
    off = hdr
    for li, (ni, no) in enumerate(zip(so.LAYER_IN, so.LAYER_OUT)):
        blob[off:off + 2 * ni * no] = bytes(2 * ni * no)  # bf16 zeros
        off += 2 * ni * no
        bias = np.zeros(no, np.float32)
        if li == len(so.LAYER_IN) - 1:
            bias[cls] = 1.0
        blob[off:off + 4 * no] = bias.tobytes()
        off += 4 * no
    assert off == len(blob)
    return bytes(blob)


@pytest.mark.parametrize("layout", ["plain", "hub", "degree", "csr"])
def test_auto_first_call_uses_default_then_prediction(cc, layout):
    """The first CC_ORDER_AUTO call of a handle solves with C-2 while the
    feature pass runs on a side stream; the next call uses the class the
    model predicts from exactly the features cc_graph_features returns."""
    rng = np.random.default_rng(21)
    cc.cc_sched_load(_random_blob(rng))
    try:
        n, s, d = GRAPHS["rmat16-sampled"]()
        want = oracle.uf_labels(n, s, d)
        if layout == "csr":
            off, cols = gg.to_csr(n, s, d)
            g = cc.cc_init(n, off.cuda(), cols.cuda(), m=cols.numel(), id_bits=32, layout=cc.CC_CSR_NATIVE,
                           on_device=True)
        else:
            g = cc.cc_init(n, s.cuda(), d.cuda())
            if layout != "plain":
                cc.cc_graph_reorder(g, cc.CC_REORDER_HUB if layout == "hub" else cc.CC_REORDER_DEGREE)
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        st = cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        assert (st.order, st.mode, st.check_interval) == (2, cc.CC_ASYNC, 1)
        assert np.array_equal(out.cpu().numpy(), want)
        out.fill_(-1)
        st2 = cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        assert np.array_equal(out.cpu().numpy(), want)
        cls, _ = cc.cc_sched_predict(cc.cc_graph_features(g))
        assert (st2.order, st2.mode, st2.check_interval) == cc.cc_sched_decode(int(cls[0]))
        cc.cc_free(g)
        # a handle freed while its feature pass may still run
        g = cc.cc_init(n, s.cuda(), d.cuda())
        cc.cc_run(g, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        cc.cc_free(g)
    finally:
        cc.cc_sched_load(None)


def test_batch_weights_take_precedence(cc):
    """cc_sched_load_batch installs the weights batched solves use; without
    them a batch uses the single-graph weights.  Synchronous sweep counts are
    deterministic, so the schedule each graph ran is visible in them."""
    vo, eo, s, d, _ = gg.batch_mix(24, seed=22, device="cuda", n_lo=300, n_hi=3e4)
    b = cc.cc_batch_init(vo, eo, s, d)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    o2, _ = cc.cc_batch_run(b, out, 2, cc.CC_SYNC, 1)
    ref = out.clone()
    o4, _ = cc.cc_batch_run(b, out, 4, cc.CC_SYNC, 1)
    assert not np.array_equal(o2, o4)
    try:
        cc.cc_sched_load(_constant_blob(6))        # order 4, synchronous
        cc.cc_sched_load_batch(_constant_blob(0))  # order 2, synchronous
        x = cc.cc_batch_features(b)
        assert (cc.cc_sched_predict(x)[0] == 6).all() and (cc.cc_sched_predict_batch(x)[0] == 0).all()
        sw, _ = cc.cc_batch_run(b, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        assert np.array_equal(sw, o2) and torch.equal(out, ref)
        cc.cc_sched_load_batch(None)
        sw, _ = cc.cc_batch_run(b, out, cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0)
        assert np.array_equal(sw, o4) and torch.equal(out, ref)
    finally:
        cc.cc_sched_load(None)
        cc.cc_sched_load_batch(None)
        cc.cc_batch_free(b)
