"""GPU parity of the learned order-5 proposer's kernels.

Score tables against the oracle's MI; unranking, candidate enumeration,
table lookup and top-k against plain enumerations; the network's forward
pass, gradients and AdamW steps against the float64 reference network
(oracle/mlp.py), with and without the library's BF16 storage rounding.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

from oracle import mlp as M
from oracle import oracle as O
from tests.helpers import F32_RTOL, random_data

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def epi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_02460_gb300 import epi as E
    E.load()
    return E


@pytest.fixture(scope="module")
def ctx(epi):
    return epi.Context(0)


@pytest.fixture(scope="module")
def small(epi, ctx):
    # 23 SNPs x 700 samples: every table of orders 1..5 fits the oracle
    geno, pheno = random_data(23, 700, seed=41)
    ds = epi.Dataset(ctx, geno, pheno)
    return geno, pheno, ds


def _oracle_all(geno, pheno, k):
    n, m = geno.shape
    combs = np.array(list(itertools.combinations(range(n), k)), dtype=np.int32)
    t = O.tables(geno, pheno, combs)
    return combs, np.array([O.mi(x[0], x[1], m) for x in t])


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_score_all_matches_oracle(epi, small, k):
    geno, pheno, ds = small
    s = epi.score_all(ds, k).cpu().numpy().astype(np.float64)
    combs, want = _oracle_all(geno, pheno, k)
    assert s.shape == want.shape
    # lexicographic order: index r is the r-th combination
    for r in (0, 1, len(combs) // 2, len(combs) - 1):
        assert O.rank(geno.shape[0], k, combs[r]) == r
    err = np.abs(s - want)
    assert (err <= F32_RTOL * want + 1e-12).all(), err.max()


def test_score_all_ragged_sizes(epi, ctx):
    # samples not a multiple of any word or tile size; one class small
    geno, pheno = random_data(17, 389, seed=5, m1=37)
    ds = epi.Dataset(ctx, geno, pheno)
    for k in (2, 3):
        s = epi.score_all(ds, k).cpu().numpy().astype(np.float64)
        _, want = _oracle_all(geno, pheno, k)
        assert (np.abs(s - want) <= F32_RTOL * want + 1e-12).all()


def test_unrank_matches_oracle(epi, ctx):
    import torch
    rng = np.random.default_rng(3)
    geno, pheno = random_data(2000, 64, seed=9)
    ds = epi.Dataset(ctx, geno, pheno)
    for k in (1, 3, 5):
        total = O.binom(2000, k)
        ranks = np.unique(np.concatenate([[0, total - 1], rng.integers(0, total, 500, dtype=np.int64)]))
        got = epi.unrank(ds, k, torch.from_numpy(ranks).cuda()).cpu().numpy()
        want = np.array([O.unrank(2000, k, int(r)) for r in ranks])
        assert (got == want).all()


def _features_cpu(mi_by_order, n, comb, orders=(1, 2, 3)):
    f = []
    for k in orders:
        vals = [mi_by_order[k][O.rank(n, k, c)] for c in itertools.combinations(comb, k)]
        vals = np.sort(np.log(np.maximum(np.array(vals), 0.0) + 1e-7))[::-1]
        f.extend(vals)
    return np.array(f)


@pytest.mark.parametrize("quad", [False, True])
def test_features5_match_oracle_scores(epi, small, quad):
    import torch
    geno, pheno, ds = small
    n = geno.shape[0]
    orders = (1, 2, 3, 4) if quad else (1, 2, 3)
    tabs = [epi.score_all(ds, k) for k in orders]
    mi = {k: _oracle_all(geno, pheno, k)[1] for k in orders}
    rng = np.random.default_rng(11)
    combs = np.array([np.sort(rng.choice(n, 5, replace=False)) for _ in range(300)], dtype=np.int32)
    cd = torch.from_numpy(combs).cuda()
    X = epi.features5(ds, *tabs[:3], cd, s4=tabs[3] if quad else None).cpu().numpy().astype(np.float64)
    want = np.stack([_features_cpu(mi, n, c, orders) for c in combs])
    assert X.shape == (300, 30 if quad else 25)
    # the kernels take logs with the hardware approximation (|error| about
    # 2^-21 relative to the log's magnitude, < 2e-5 here)
    np.testing.assert_allclose(X, want, rtol=0, atol=2e-5)
    # each group is sorted descending
    for lo, hi in ((0, 5), (5, 15), (15, 25)) + (((25, 30),) if quad else ()):
        assert (np.diff(X[:, lo:hi], axis=1) <= 0).all()


def _candidate_space(n, triples):
    out = []
    for t in triples:
        rest = [s for s in range(n) if s not in t]
        for u, v in itertools.combinations(rest, 2):
            out.append(sorted(list(t) + [u, v]))
    return np.array(out, dtype=np.int32)


def test_candidates5_enumeration_and_keep(epi, small):
    import torch
    geno, pheno, ds = small
    n = geno.shape[0]
    s3 = epi.score_all(ds, 3)
    s3h = s3.cpu().numpy()
    triples = np.array([[0, 1, 2], [3, 9, 20], [1, 2, 7], [0, 2, 21], [5, 6, 22]], dtype=np.int32)
    want = _candidate_space(n, triples)
    tri_d = torch.from_numpy(triples).cuda()
    got, keep = epi.candidates5(ds, tri_d, 0, len(want), s3=s3)
    assert (got.cpu().numpy() == want).all()
    # ragged sub-range
    sub = epi.candidates5(ds, tri_d, 101, 333)
    assert (sub.cpu().numpy() == want[101:434]).all()
    # keep: the generating triple is the best of the set's ten triples
    per = math.comb(n - 3, 2)
    keep = keep.cpu().numpy()
    for i in range(len(want)):
        t = tuple(triples[i // per])
        key = lambda c: (-s3h[O.rank(n, 3, c)], O.rank(n, 3, c))
        best = min(itertools.combinations(want[i], 3), key=key)
        assert keep[i] == (1 if tuple(best) == t else 0)
    # every distinct set of the space is kept exactly once when its best
    # triple is listed
    kept = {tuple(c) for c, k in zip(want, keep) if k}
    assert sum(keep) == len(kept)


@pytest.mark.parametrize("n,m,m1,count", [(23, 700, None, 1), (23, 700, None, 1001), (12, 64, 32, 50),
                                           (30, 5000, 1500, 777), (40, 9000, 6300, 300), (9, 2100, 2100, 40)])
def test_score5_matches_oracle(epi, ctx, n, m, m1, count):
    """The fused order-5 FP32 scorer (tables counted in registers): within
    1e-6 relative of the oracle's FP64 MI, on sample counts that span one
    and several 64-word chunks with the case/control split inside a chunk,
    unbalanced and single-class phenotypes, and a ragged number of sets."""
    import torch
    geno, pheno = random_data(n, m, seed=n * 7 + count, m1=m1)
    ds = epi.Dataset(ctx, geno, pheno)
    rng = np.random.default_rng(count)
    combs = np.array([np.sort(rng.choice(n, 5, replace=False)) for _ in range(count)], dtype=np.int32)
    got = epi.score5(ds, torch.from_numpy(combs).cuda()).cpu().numpy().astype(np.float64)
    t = O.tables(geno, pheno, combs)
    want = np.array([O.mi(x[0], x[1], m) for x in t])
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-12)
    # and the table path's FP32 value within the FP32 bound (2 (2*243+32) u)
    f32, _ = epi.score_tables(ds, 5, epi.tables(ds, combs))
    np.testing.assert_allclose(got, f32.astype(np.float64), rtol=2 * (2 * 243 + 32) * 2.0 ** -24, atol=1e-12)


def test_lookup_is_table_at_rank(epi, small):
    import torch
    geno, pheno, ds = small
    n = geno.shape[0]
    s5 = epi.score_all(ds, 5)
    rng = np.random.default_rng(2)
    combs = np.array([np.sort(rng.choice(n, 5, replace=False)) for _ in range(257)], dtype=np.int32)
    got = epi.lookup(ds, 5, s5, torch.from_numpy(combs).cuda()).cpu().numpy()
    s5h = s5.cpu().numpy()
    want = np.array([s5h[O.rank(n, 5, c)] for c in combs])
    assert (got == want).all()


@pytest.mark.parametrize("count,k", [(1, 1), (100, 4096), (1_000_003, 100), (2_500_000, 4096), (70_000, 1000)])
def test_topk_matches_sort(epi, ctx, count, k):
    import torch
    rng = np.random.default_rng(count + k)
    # few distinct values: many ties broken by index
    v = rng.integers(0, 50, count).astype(np.float32) * np.float32(0.25)
    keep = (rng.random(count) < 0.7).astype(np.uint8)
    vals, idx = epi.topk(ctx, torch.from_numpy(v).cuda(), k, keep=torch.from_numpy(keep).cuda())
    cand = np.nonzero(keep)[0]
    order = cand[np.lexsort((cand, -v[cand]))][:k]
    assert (idx.cpu().numpy() == order).all()
    assert (vals.cpu().numpy() == v[order]).all()
    vals, idx = epi.topk(ctx, torch.from_numpy(v).cuda(), k)
    order = np.lexsort((np.arange(count), -v))[:k]
    assert (idx.cpu().numpy() == order).all()


def test_topk_skips_nan_keeps_neg_inf(epi, ctx):
    import torch
    v = np.array([np.nan, -np.inf, 1.0, np.nan, 0.5, -np.inf], dtype=np.float32)
    vals, idx = epi.topk(ctx, torch.from_numpy(v).cuda(), 6)
    assert list(idx.cpu().numpy()) == [2, 4, 1, 5]


def _bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _net_inputs(rows, n_in, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-9.0, -1.0, (rows, n_in)).astype(np.float32)
    t = rng.normal(-2.0, 0.5, rows).astype(np.float32)
    return X, t


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("rows,hidden", [(1, 64), (300, 64), (1000, 256)])
def test_mlp_gradients_match_reference(epi, ctx, rows, hidden):
    import torch
    net = epi.MLP(ctx, 25, hidden, seed=7)
    theta = net.params().astype(np.float64)
    X, t = _net_inputs(rows, 25, rows)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    y = net.forward(Xd).cpu().numpy().astype(np.float64)
    g, loss = net.gradients(Xd, td)
    g = g.astype(np.float64)
    # same storage rounding as the library: agreement up to FP32 accumulation
    y_q, _ = M.forward(theta, X, 25, hidden, rnd=_bf16)
    g_q = M.gradients(theta, X, t, 25, hidden, rnd=_bf16, rnd_dz=_bf16)
    assert _rel(y, y_q) <= 1e-4
    offs = np.cumsum([0, hidden * 25, hidden, hidden * hidden, hidden, hidden, 1])
    for a, b in zip(offs[:-1], offs[1:]):
        assert _rel(g[a:b], g_q[a:b]) <= 2e-3, (a, b, _rel(g[a:b], g_q[a:b]))
    assert abs(loss - M.loss(theta, X, t, 25, hidden, rnd=_bf16)) <= 1e-4 * abs(loss) + 1e-7
    # plain float64 network: every prediction within the BF16 rounding of the
    # sum of absolute products feeding it (the output is a difference of much
    # larger terms) ...
    y_64, (_, _, _, _, H2, _, W3) = M.forward(theta, X, 25, hidden)
    scale = np.abs(H2) @ np.abs(W3) + 1.0
    assert (np.abs(y - y_64) <= 2.0 ** -6 * scale).all()
    # ... and, over a batch, gradients at targets well away from the
    # predictions within a few BF16 roundings
    if rows >= 300:
        t2 = (y_64 + scale).astype(np.float32)
        g2, _ = net.gradients(Xd, torch.from_numpy(t2).cuda())
        g_64 = M.gradients(theta, X, t2, 25, hidden)
        assert _rel(g2.astype(np.float64), g_64) <= 3e-2
    net.close()


def _grad_magnitudes(theta, X, t, n_in, h, rnd):
    """Per gradient element: S, the sum of the absolute values of its terms
    (the same chain rule with every factor replaced by its absolute value);
    L, its largest single term; and A, the part of S that passes through ReLU
    masks whose pre-activation lies within float32 rounding of zero (where the
    library's float32 sum and the float64 reference may disagree about the
    sign)."""
    W1, b1, W2, b2, W3, b3 = M.unpack(np.asarray(theta, np.float64), n_in, h)
    W1q, W2q, W3q = rnd(W1), rnd(W2), rnd(W3)
    Xq = np.abs(rnd(np.asarray(X, np.float64)))
    Z1 = rnd(np.asarray(X, np.float64)) @ W1q.T + b1
    S_z1 = Xq @ np.abs(W1q.T) + np.abs(b1)
    H1 = rnd(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2q.T + b2
    S_z2 = H1 @ np.abs(W2q.T) + np.abs(b2)
    H2 = rnd(np.maximum(Z2, 0.0))
    y = H2 @ W3q + b3[0]
    B = X.shape[0]
    dy = np.abs(2.0 * (y - np.asarray(t, np.float64)) / B)
    amb1 = np.abs(Z1) <= 1e-5 * S_z1
    amb2 = np.abs(Z2) <= 1e-5 * S_z2
    on1, on2 = (Z1 > 0) | amb1, (Z2 > 0) | amb2
    D2 = np.outer(dy, np.abs(W3q)) * on2            # |dZ2| (ambiguous entries counted)
    D2a = np.outer(dy, np.abs(W3q)) * amb2
    D1 = (D2 @ np.abs(W2q)) * on1
    D1a = (D2a @ np.abs(W2q)) * on1 + (D2 @ np.abs(W2q)) * amb1

    def outer_max(P, Q):                            # max over rows b of P[b, i] Q[b, j]
        out = np.zeros((P.shape[1], Q.shape[1]))
        for b0 in range(0, P.shape[0], 64):
            blk = P[b0:b0 + 64, :, None] * Q[b0:b0 + 64, None, :]
            out = np.maximum(out, blk.max(axis=0))
        return out

    S = np.concatenate([(D1.T @ Xq).ravel(), D1.sum(0), (D2.T @ H1).ravel(), D2.sum(0), H2.T @ dy, [dy.sum()]])
    L = np.concatenate([outer_max(D1, Xq).ravel(), D1.max(0), outer_max(D2, H1).ravel(), D2.max(0),
                        (H2 * dy[:, None]).max(0), [dy.max()]])
    A = np.concatenate([(D1a.T @ Xq).ravel(), D1a.sum(0), (D2a.T @ H1).ravel(), D2a.sum(0),
                        np.zeros(h), [0.0]])
    return S, L, A


@pytest.mark.parametrize("rows,hidden", [(1, 64), (300, 64), (1000, 256)])
def test_mlp_gradients_elementwise(epi, ctx, rows, hidden):
    """Every gradient element against the float64 reference with the
    library's BF16 storage points.  Both compute the same chain rule on the
    same rounded operands; they differ by float32 accumulation (at most about
    K 2^-24 S_i for K summed terms), by a stored BF16 activation that rounds to
    the neighbouring value when its float32 and float64 pre-images straddle a
    rounding boundary (one term off by at most 2^-7 of itself), and by ReLU
    masks at pre-activations within rounding of zero.  Hence, per element i
    with S_i the sum of the absolute values of its terms, L_i the largest
    term and A_i the part through such masks:
        |g_i - g_ref,i| <= 2^-6 L_i + 2^-12 S_i + A_i.
    A wrong element (a dropped term, a wrong sign, a missing bias row) moves
    g_i by a whole term or by g_i itself, beyond that bound except under
    extreme cancellation; the median relative error must also stay at
    float32 level."""
    import torch
    net = epi.MLP(ctx, 25, hidden, seed=11)
    theta = net.params().astype(np.float64)
    X, _ = _net_inputs(rows, 25, rows + 5)
    # targets away from the predictions, so that dy = 2 (y - t) / B has no
    # cancellation of its own
    y_q, (_, _, _, _, H2, _, W3) = M.forward(theta, X, 25, hidden, rnd=_bf16)
    scale = np.abs(H2) @ np.abs(W3) + 1.0
    t = (y_q + 4.0 * scale * np.where(np.arange(rows) % 2 == 0, 1.0, -1.0)).astype(np.float32)
    g, _ = net.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    g = g.astype(np.float64)
    g_q = M.gradients(theta, X, t, 25, hidden, rnd=_bf16, rnd_dz=_bf16)
    S, L, A = _grad_magnitudes(theta, X, t, 25, hidden, _bf16)
    err = np.abs(g - g_q)
    bound = 2.0 ** -6 * L + 2.0 ** -12 * S + A + 1e-30
    worst = int(np.argmax(err / bound))
    assert (err <= bound).all(), (worst, g[worst], g_q[worst], S[worst], L[worst], A[worst])
    nz = np.abs(g_q) > 1e-3 * S
    assert np.median(err[nz] / np.abs(g_q[nz])) <= 1e-4
    net.close()


def test_mlp_adamw_steps_match_reference(epi, ctx):
    import torch
    h = 64
    net = epi.MLP(ctx, 25, h, seed=3)
    theta = net.params().astype(np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    X, t = _net_inputs(513, 25, 1)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    lr, wd = 3e-3, 1e-2
    for step in (1, 2, 3):
        g, _ = net.gradients(Xd, td)          # the gradient the step will use
        net.train_step(Xd, td, lr, wd)
        theta, m, v = M.adamw_step(theta, g.astype(np.float64), m, v, step, lr, wd)
        got = net.params().astype(np.float64)
        np.testing.assert_allclose(got, theta, rtol=2e-6, atol=2e-8)
        theta = got
    net.close()


def test_mlp_training_reduces_loss(epi, ctx):
    import torch
    rng = np.random.default_rng(0)
    X = rng.uniform(-4, 0, (4096, 25)).astype(np.float32)
    t = (X[:, 15:25].mean(axis=1) * 0.5 + np.sin(X[:, 0])).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    net = epi.MLP(ctx, 25, 128, seed=1)
    first = net.train_step(Xd, td, 1e-3, 0.0)
    for _ in range(300):
        last = net.train_step(Xd, td, 1e-3, 0.0)
    assert last < 0.05 * first


def test_mlp_save_load_roundtrip(epi, ctx, tmp_path):
    import torch
    a = epi.MLP(ctx, 25, 32, seed=5)
    b = epi.MLP(ctx, 25, 32, seed=6)
    p = str(tmp_path / "net.bin")
    a.save(p)
    b.load_file(p)
    assert (a.params() == b.params()).all()
    X, _ = _net_inputs(77, 25, 9)
    Xd = torch.from_numpy(X).cuda()
    assert torch.equal(a.forward(Xd), b.forward(Xd))
    c = epi.MLP(ctx, 25, 64, seed=5)
    with pytest.raises(ValueError):
        c.load_file(p)


@pytest.mark.parametrize("cols", [25, 30])
def test_heuristic5_is_sum_of_top_order_features(epi, ctx, cols):
    import torch
    X, _ = _net_inputs(1001, cols, 4)
    got = epi.heuristic5(ctx, torch.from_numpy(X).cuda()).cpu().numpy()
    lo = 15 if cols == 25 else 25
    np.testing.assert_allclose(got, X[:, lo:cols].astype(np.float64).sum(axis=1), rtol=1e-6)


@pytest.mark.parametrize("rows,n_in", [(1, 25), (127, 25), (128, 25), (129, 25), (1000, 25), (70001, 25),
                                      (70001, 30), (3001, 32), (385, 1), (1000, 16), (1000, 17)])
def test_mlp_tensor_core_forward_matches_reference(epi, ctx, rows, n_in):
    import torch
    net = epi.MLP(ctx, n_in, 256, seed=rows)
    rng = np.random.default_rng(rows + n_in)
    shift = rng.uniform(-6, -3, n_in).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, n_in).astype(np.float32)
    net.set_input_norm(shift, scale)
    theta = net.params().astype(np.float64)
    theta[n_in * 256:n_in * 256 + 256] = rng.normal(0, 0.1, 256)      # nonzero b1
    net.set_params(theta.astype(np.float32))
    theta = net.params().astype(np.float64)
    X, _ = _net_inputs(rows, n_in, rows + 1)
    Xd = torch.from_numpy(X).cuda()
    net.set_forward_path("tensor_cores")
    y_tc = net.forward(Xd).cpu().numpy().astype(np.float64)
    net.set_forward_path("cuda_cores")
    y_cc = net.forward(Xd).cpu().numpy().astype(np.float64)
    Xn = (X - shift) * scale                                            # float32, as the kernels form it
    y_q, (_, _, _, _, H2, _, W3) = M.forward(theta, Xn, n_in, 256, rnd=_bf16)
    bound = 2.0 ** -7 * (np.abs(H2) @ np.abs(W3) + 1.0)
    # both paths round the hidden layers to BF16 at the reference's points;
    # a different FP32 accumulation order may move a rounded activation by
    # one BF16 ulp, so each prediction is held to the rounding of the
    # absolute products feeding it, and the batch to 1e-3 norm-wise
    for y in (y_tc, y_cc):
        assert _rel(y, y_q) <= 1e-3
        assert (np.abs(y - y_q) <= bound).all()


def test_mlp_tensor_core_path_needs_its_shape(epi, ctx):
    with pytest.raises(epi.EpiError):
        epi.MLP(ctx, 25, 64).set_forward_path("tensor_cores")
    with pytest.raises(epi.EpiError):
        epi.MLP(ctx, 33, 256).set_forward_path("tensor_cores")
