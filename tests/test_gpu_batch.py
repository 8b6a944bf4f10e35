"""Batched fused launch (hc_batch_*) against the oracle (needs a GPU).

Many fields of uneven shapes and block sizes, each with its own operations,
run in one persistent kernel: statistics must equal the oracle's exact sums,
integer stencil numerators must equal the oracle's bit for bit, and float
outputs must agree within the stated tolerances.  The launch must also be
repeatable: graph replays, launch shapes (threads, tile height, unit size)
and repeated runs give identical bytes, and every launch leaves its
workspace zeroed.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_25206_gb300 import hc

    hc.lib()
    return hc, torch, torch.device("cuda:0")


# (shape, S, ops, eb, rel, seed)
MIXED = [
    ((40, 33, 70), 32, "mean|variance|laplacian", 1e-3, True, 11),
    ((17, 64, 64), 16, "variance", 1e-3, True, 12),
    ((9, 130, 37), 64, "mean|laplacian", 1e-2, True, 13),
    ((300, 257), 128, "variance|laplacian", 1e-3, True, 14),
    ((5000,), 32, "mean|variance|laplacian", 1e-3, True, 15),
    ((3, 5, 7), 32, "mean|variance", 1e-4, True, 16),
    ((64, 48, 100), 100, "laplacian", 1e-3, True, 17),
    ((1, 1, 1), 32, "mean|variance|laplacian", 1e-3, True, 18),
    ((33, 31, 29), 7, "variance|laplacian", 1e-3, True, 19),
    ((8, 8, 4096), 32, "mean|variance", 1e-3, True, 20),
]


def _field(shape, seed):
    import synth

    if int(np.prod(shape)) < 64:
        return np.random.default_rng(seed).random(shape).astype(np.float32)
    return synth.grf_field(shape, seed)


def _make(env, orc, specs, field_dtype="int64", **tune):
    hc, torch, dev = env
    items, refs = [], []
    for shape, S, ops, eb, rel, seed in specs:
        x = _field(shape, seed)
        ref, eps = orc.compress(x, eb, rel, S)
        c = hc.compress(torch.from_numpy(x).to(dev), eb, rel=rel, S=S)
        assert np.array_equal(c.stream[: c.nbytes].cpu().numpy(), ref)
        items.append((c, ops))
        refs.append((orc.decode(ref, "q"), eps, ops))
    return hc.Batch(items, field_dtype=field_dtype, **tune), refs


def _check(orc, batch, refs, field_dtype):
    for (sc, f), (q, eps, ops) in zip(batch.results(), refs):
        s1, s2 = orc.sums_q(q)
        if "mean" in ops or "variance" in ops:
            assert sc["status"] == 0
            assert sc["n"] == q.size and sc["s1"] == s1
            m_ref, v_ref, _ = orc.finalize(q.size, s1, s2, eps)
            assert abs(sc["mean"] - m_ref) <= 1e-12 * max(abs(m_ref), eps)
            if "variance" in ops:
                assert sc["s2"] == s2
                if q.size >= 2:
                    assert abs(sc["variance"] - v_ref) <= 1e-12 * max(v_ref, (2 * eps) ** 2)
        if "laplacian" in ops:
            got = f.cpu().numpy()
            if field_dtype == "int64":
                assert np.array_equal(got, orc.lap_q(q))
            else:
                val = orc.stencil_q(q, orc.KIND_LAPLACIAN, eps)
                tol = 1e-6 if field_dtype == "float32" else 1e-12
                assert np.all(np.abs(got - val) <= tol * np.maximum(np.abs(val), 2 * eps))


@pytest.mark.parametrize("field_dtype", ["int64", "float32", "float64"])
def test_mixed_batch_matches_oracle(env, orc, field_dtype):
    hc, torch, dev = env
    b, refs = _make(env, orc, MIXED, field_dtype=field_dtype)
    b.run()
    torch.cuda.synchronize()
    assert b.status() == 0
    _check(orc, b, refs, field_dtype)
    assert int(b.ws.count_nonzero()) == 0  # the launch left its workspace zeroed


def test_batch_equals_single_field_calls(env, orc):
    """Same bytes as the one-field entry points (Laplacian int64 and float32,
    exact sums)."""
    hc, torch, dev = env
    for fd in ("int64", "float32"):
        b, refs = _make(env, orc, MIXED, field_dtype=fd)
        b.run()
        for c, spec, (sc, f) in zip(b.comps, MIXED, b.results()):
            ops = spec[2]
            if "laplacian" in ops:
                one = hc.laplacian(c, out_dtype=fd)
                assert torch.equal(one, f)
            if "variance" in ops:
                r = hc.parse_scalar(hc.variance(c, level="q"))
                assert (r["s1"], r["s2"]) == (sc["s1"], sc["s2"])
                assert r["variance"] == sc["variance"] or (np.isnan(r["variance"]) and np.isnan(sc["variance"]))


def test_other_field_ops(env, orc):
    hc, torch, dev = env
    # block 32 rows of 40 (8 outputs per item), 36 (4) and 30 (1) codes take
    # the pipelined tile; block 64 the general one
    specs = [((20, 30, 40), 32, "gradmag|variance", 1e-3, True, 31), ((50, 70), 64, "gradmag", 1e-3, True, 32),
             ((10, 12, 36), 32, "gradmag|mean", 1e-3, True, 35), ((14, 22, 30), 32, "gradmag", 1e-3, True, 36)]
    b, refs = _make(env, orc, specs, field_dtype="float64")
    b.run()
    for (sc, f), (q, eps, ops) in zip(b.results(), refs):
        val = orc.stencil_q(q, orc.KIND_GRADMAG, eps)
        assert np.all(np.abs(f.cpu().numpy() - val) <= 1e-12 * np.maximum(np.abs(val), eps))
    for ax in range(3):
        specs = [((20, 30, 40), 32, "derivative|mean", 1e-3, True, 33), ((12, 9, 300), 16, "derivative", 1e-3, True, 34),
                 ((10, 12, 36), 32, "derivative|variance", 1e-3, True, 37), ((14, 22, 30), 32, "derivative", 1e-3, True, 38)]
        b, refs = _make(env, orc, specs, field_dtype="int64", axis=ax)
        b.run()
        for (sc, f), (q, eps, ops) in zip(b.results(), refs):
            assert np.array_equal(f.cpu().numpy(), orc.deriv_q(q, ax))
            if sc is not None:
                assert (sc["s1"], sc["s2"] if "variance" in ops else 0) == \
                    (orc.sums_q(q)[0], orc.sums_q(q)[1] if "variance" in ops else 0)


# Rows whose length is not a multiple of 4 (block 32) take the padded ring:
# one to several 8-wide items per row, the last one partial; tiles of one row
# up to the whole plane (ty caps the height); 3-D, 2-D and 1-D fields.
PADDED_3D = [(3, 4, 7), (5, 9, 9), (4, 6, 15), (3, 17, 23), (6, 5, 33), (2, 3, 63), (7, 2, 2), (2, 1, 129),
             (9, 13, 37), (30, 70, 131), (1, 1, 1), (1, 6, 5)]
PADDED_LOW = [(7, 13), (11, 3), (5,), (3001,), (40, 257)]


@pytest.mark.parametrize("ty", [0, 1, 2])
def test_padded_rows_every_operation(env, orc, ty):
    hc, torch, dev = env
    tune = {"ty": ty} if ty else {}
    shapes = PADDED_3D + PADDED_LOW
    specs = [(sh, 32, "laplacian|variance", 1e-3, True, 60 + j) for j, sh in enumerate(shapes)]
    for fd in ("int64", "float32", "float64"):
        b, refs = _make(env, orc, specs, field_dtype=fd, **tune)
        b.run()
        torch.cuda.synchronize()
        assert b.status() == 0
        _check(orc, b, refs, fd)
        for c, (sc, f) in zip(b.comps, b.results()):
            assert torch.equal(hc.laplacian(c, out_dtype=fd), f), (fd, c.shape)
    specs = [(sh, 32, "gradmag|mean", 1e-3, True, 90 + j) for j, sh in enumerate(shapes)]
    b, refs = _make(env, orc, specs, field_dtype="float64", **tune)
    b.run()
    for (sc, f), (q, eps, ops) in zip(b.results(), refs):
        assert sc["s1"] == orc.sums_q(q)[0]
        val = orc.stencil_q(q, orc.KIND_GRADMAG, eps)
        assert np.all(np.abs(f.cpu().numpy() - val) <= 1e-12 * np.maximum(np.abs(val), eps))
    for ax in range(3):
        specs = [(sh, 32, "derivative|variance", 1e-3, True, 120 + j) for j, sh in enumerate(PADDED_3D)]
        b, refs = _make(env, orc, specs, field_dtype="int64", axis=ax, **tune)
        b.run()
        for (sc, f), (q, eps, ops) in zip(b.results(), refs):
            assert np.array_equal(f.cpu().numpy(), orc.deriv_q(q, ax)), (ax, q.shape)
            assert (sc["s1"], sc["s2"]) == orc.sums_q(q)
    for ax in range(2):
        specs = [(sh, 32, "derivative", 1e-3, True, 150 + j) for j, sh in enumerate(PADDED_LOW) if len(sh) == 2]
        b, refs = _make(env, orc, specs, field_dtype="float32", axis=ax, **tune)
        b.run()
        for (sc, f), (q, eps, ops) in zip(b.results(), refs):
            val = orc.stencil_q(q, orc.KIND_DERIV, eps, axis=ax)
            assert np.all(np.abs(f.cpu().numpy() - val) <= 1e-6 * np.maximum(np.abs(val), eps)), (ax, q.shape)


def test_graph_replay_and_launch_shapes_identical(env, orc):
    hc, torch, dev = env
    b, refs = _make(env, orc, MIXED, field_dtype="float32")
    b.run()
    torch.cuda.synchronize()
    base_f = [f.clone() if f is not None else None for f in b.fields]
    base_s = b.scalars.clone()
    for f in b.fields:
        if f is not None:
            f.zero_()
    b.scalars.zero_()
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.scalars, base_s)
    for f, g in zip(b.fields, base_f):
        if f is not None:
            assert torch.equal(f, g)
    assert int(b.ws.count_nonzero()) == 0
    b.close()
    for tune in ({"threads": 128}, {"threads": 512}, {"ty": 2}, {"unit_elems": 1}, {"ctas_per_sm": 1}):
        b2, _ = _make(env, orc, MIXED, field_dtype="float32", **tune)
        b2.run()
        torch.cuda.synchronize()
        assert torch.equal(b2.scalars, base_s), tune
        for f, g in zip(b2.fields, base_f):
            if f is not None:
                assert torch.equal(f, g), tune


def test_corrupt_item_reported_others_correct(env, orc):
    hc, torch, dev = env
    import synth

    x = synth.grf_field((16, 16, 64), 4)
    ref, eps = orc.compress(x, 1e-3, True, 32)
    bad = ref.copy()
    bad[256 + 100] = 31  # disagrees with the chunk index
    cb = hc.from_stream(torch.from_numpy(bad).to(dev))
    y = synth.grf_field((20, 20, 20), 5)
    ref2, eps2 = orc.compress(y, 1e-3, True, 32)
    cg = hc.compress(torch.from_numpy(y).to(dev), 1e-3, rel=True, S=32)
    b = hc.Batch([(cb, "variance|laplacian"), (cg, "variance|laplacian")], field_dtype="int64")
    b.run()
    torch.cuda.synchronize()
    (s_bad, _), (s_good, f_good) = b.results()
    assert s_bad["status"] == hc.HC_ERR_CORRUPT
    q2 = orc.decode(ref2, "q")
    assert s_good["status"] == 0 and (s_good["s1"], s_good["s2"]) == orc.sums_q(q2)
    assert np.array_equal(f_good.cpu().numpy(), orc.lap_q(q2))
    assert b.status() == hc.HC_ERR_CORRUPT
    assert b.status() == 0
    assert int(b.ws.count_nonzero()) == 0


@pytest.fixture(scope="module")
def batched_fields():
    import synth

    shapes = synth.log_uniform_shapes(64, 32, 384, 3)
    return [synth.grf_field(shape, 3000 + j) for j, shape in enumerate(shapes)]


@pytest.mark.parametrize("S", [16, 32, 64, 128])
def test_batched_config_full_size(env, orc, batched_fields, S):
    """64 float32 fields, every axis drawn log-uniformly from [32, 384]
    (seed 3), k^-3 field plus 5% spikes, value-range-relative eb = 1e-3:
    mean, variance and Laplacian in one launch.  Exact sums for every field;
    the Laplacian numerators at sampled points of every field."""
    hc, torch, dev = env
    items, refs = [], []
    for x in batched_fields:
        shape = x.shape
        ref, eps = orc.compress(x, 1e-3, True, S)
        c = hc.compress(torch.from_numpy(x).to(dev), 1e-3, rel=True, S=S)
        assert c.nbytes == ref.size
        items.append((c, "mean|variance|laplacian"))
        refs.append((ref, eps, shape))
    b = hc.Batch(items, field_dtype="int64")
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    assert b.status() == 0
    rng = np.random.default_rng(S)
    for (sc, f), (ref, eps, shape) in zip(b.results(), refs):
        q = orc.decode(ref, "q")
        s1, s2 = orc.sums_q(q)
        assert (sc["s1"], sc["s2"]) == (s1, s2)
        idx = np.unique(np.concatenate([[0, q.size - 1], rng.integers(0, q.size, 2000)]))
        num, _ = orc.stencil_at(q, orc.KIND_LAPLACIAN, eps, idx)
        assert np.array_equal(f.reshape(-1)[torch.from_numpy(idx).to(dev)].cpu().numpy(), num)
    assert int(b.ws.count_nonzero()) == 0
    b.close()


def _vector_components(orc, hc, torch, dev, shape, S, rel, seed, predictor="delta"):
    import synth

    comps, qs, eps = [], [], []
    pred = 1 if predictor == "mean" else 0
    for c in range(len(shape)):
        x = synth.grf_field(shape, seed + c)
        ref, e = orc.compress(x, 1e-3 if rel else 2e-3, rel, S, pred=pred)
        comps.append(hc.from_stream(torch.from_numpy(ref).to(dev)))
        qs.append(orc.decode(ref, "q"))
        eps.append(e)
    return comps, qs, eps


@pytest.mark.parametrize("field_dtype", ["float64", "float32", "int64"])
def test_vector_items_in_a_mixed_batch(env, orc, field_dtype):
    """Divergence and curl items (Section V-C) in one batch with scalar items:
    each vector output equals hc_op_divergence / hc_op_curl on the same
    components bit for bit, and the oracle's (exact integer numerators for
    int64; float64 values bit for bit; float32 within 1e-6 of the field's
    scale); the scalar items keep their oracle results; graph replay gives
    the same outputs."""
    hc, torch, dev = env
    div3, q3, e3 = _vector_components(orc, hc, torch, dev, (10, 24, 40), 32, False, 7100)
    div2, q2, e2 = _vector_components(orc, hc, torch, dev, (33, 50), 16, False, 7200, "mean")
    curl2, qc, ec = _vector_components(orc, hc, torch, dev, (40, 64), 32, False, 7300)
    x = _field((12, 20, 48), 7400)
    ref, eps = orc.compress(x, 1e-3, True, 32)
    c = hc.from_stream(torch.from_numpy(ref).to(dev))
    q = orc.decode(ref, "q")
    b = hc.Batch([(tuple(div3), "divergence"), (c, "mean|variance|laplacian"), (tuple(div2), "divergence"),
                  (tuple(curl2), "curl")], field_dtype=field_dtype)
    for run in (b.run, lambda: (b.capture(), b.replay())):
        run()
        torch.cuda.synchronize()
        assert b.status() == 0
        res = b.results()
        for k, spec in enumerate(((div3, q3, e3, "div"), None, (div2, q2, e2, "div"), (curl2, qc, ec, "curl"))):
            if spec is None:
                continue
            comps, qs, eps_c, op = spec
            got = res[k][1].cpu().numpy()
            one = (hc.divergence if op == "div" else hc.curl)(comps, out_dtype=field_dtype).cpu().numpy()
            assert np.array_equal(got, one), (k, op)
            num, val = orc.divergence_q(qs, eps_c) if op == "div" else orc.curl2_q(qs[0], qs[1], eps_c[0], eps_c[1])
            if field_dtype == "int64":
                assert np.array_equal(got, num)
            elif field_dtype == "float64":
                assert np.array_equal(got, val)
            else:
                assert np.all(np.abs(got - val) <= 1e-6 * np.maximum(np.abs(val), min(eps_c)))
        s1, s2 = orc.sums_q(q)
        st = res[1][0]
        assert (st["s1"], st["s2"], st["status"]) == (s1, s2, 0)
        lap = res[1][1].cpu().numpy()
        if field_dtype == "int64":
            assert np.array_equal(lap, orc.lap_q(q))
    b.close()


def test_vector_item_rules(env, orc):
    hc, torch, dev = env
    comps, _, _ = _vector_components(orc, hc, torch, dev, (6, 8, 16), 32, False, 7500)
    for items, status in ((((tuple(comps), "curl"),), hc.HC_ERR_UNSUPPORTED),  # 3-D curl
                          (((tuple(comps[:2]), "divergence"),), hc.HC_ERR_INVALID_ARG),  # ncomp != ndim
                          (((tuple(comps), "divergence|mean"),), hc.HC_ERR_INVALID_ARG)):  # a second op
        with pytest.raises(hc.HcError) as e:
            hc.Batch(list(items))
        assert e.value.status == status
    cl = hc.compress(torch.from_numpy(_field((6, 8, 16), 7600)).to(dev), 1e-3, predictor="lorenzo")
    with pytest.raises(hc.HcError) as e:
        hc.Batch([((comps[0], comps[1], cl), "divergence")])
    assert e.value.status == hc.HC_ERR_UNSUPPORTED
