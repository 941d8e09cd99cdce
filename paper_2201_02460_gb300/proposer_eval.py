"""Training and recall evaluation of the learned order-5 proposer.

Trains the proposer networks (epi_proposer_train) on synthetic 200-SNP x
2000-sample datasets shaped like the training configuration (Hardy-Weinberg
genotypes, MAF ~ U[0.05, 0.5], balanced classes, every other dataset with a
planted 5-SNP parity): the 25-256-256-1 network on the order-1..3 features
and the 30-256-256-1 network that also sees the five four-way scores.  Then
measures on held-out datasets of the same shape the recall of the exhaustive
order-5 top-100 (the tensor-core search) among the proposer's top-100, for
each network and for the network-free heuristic of the same features, by
expanded triples T and re-score budget R.

    python -m paper_2201_02460_gb300.proposer_eval [--train 8] [--epochs 4] [--epochs30 2]

prints one JSON line.  Every step runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

from . import epi, synth


def make(ctx, seed: int, plant: bool, n_snps: int = 200, n_samples: int = 2000):
    d = synth.make_dataset(n_snps, n_samples // 2, n_samples - n_samples // 2, seed=seed,
                           plant_q=5 if plant else 0, plant_e=0.25 if plant else 0.0)
    return epi.Dataset(ctx, d.geno, d.pheno)


def evaluate(ctx=None, n_train: int = 8, epochs: int = 4, epochs30: int = 2, train_triples: int = 1024,
             n_eval: int = 3, budgets=(10 ** 6, 10 ** 7), eval_triples=(4096, 65536), seed: int = 7) -> dict:
    ctx = ctx or epi.Context(0)
    t0 = time.perf_counter()
    train = [make(ctx, synth.BASE_SEED + 200 + i, i % 2 == 0) for i in range(n_train)]
    evals = [make(ctx, synth.BASE_SEED + 103 + i, i % 2 == 0) for i in range(n_eval)]
    truth = []
    t_truth = time.perf_counter()
    for ds in evals:
        r = epi.search(ds, 5, 100, path="tc")
        truth.append({tuple(int(x) for x in c) for c in r.combs})
    t_truth = time.perf_counter() - t_truth
    nets, training = {}, {}
    for n_in, ep in ((25, epochs), (30, epochs30)):
        net = epi.MLP(ctx, n_in, 256, seed=1)
        t1 = time.perf_counter()
        losses = epi.proposer_train(net, train, train_triples, ep, 8192, 1e-3, 1e-4, 0.5, seed)
        training[n_in] = dict(epochs=ep, losses=[float(x) for x in losses], seconds=time.perf_counter() - t1)
        nets[n_in] = net
    rows = []
    for n_in, net in nets.items():
        for T in eval_triples:
            for R in budgets:
                for name, scorer in (("heuristic", None), ("network", net)):
                    rec, secs = [], []
                    for ds, tr in zip(evals, truth):
                        t1 = time.perf_counter()
                        r, st = epi.proposer_search(ds, scorer, T, R, 100, quad_features=n_in == 30)
                        secs.append(time.perf_counter() - t1)
                        rec.append(len({tuple(int(x) for x in c) for c in r.combs} & tr) / 100.0)
                    rows.append(dict(features=n_in, ranking=name, top_triples=T, budget=R, recall_at_100=rec,
                                     mean_recall=sum(rec) / len(rec),
                                     seconds_per_search=sum(secs[1:]) / max(len(secs) - 1, 1)))
    for net in nets.values():
        net.close()
    for ds in train + evals:
        ds.close()
    return dict(metric="top-N recall at k=5 (recall@100 of the exhaustive order-5 top-100)",
                datasets=dict(train=n_train, eval=n_eval, n_snps=200, n_samples=2000,
                              data="synthetic HWE, MAF U[0.05,0.5], every other dataset with a planted 5-SNP parity"),
                training=dict(top_triples=train_triples, batch=8192, lr=1e-3, wd=1e-4, tail_fraction=0.5,
                              by_features={str(k): v for k, v in training.items()}),
                exhaustive_seconds_per_dataset=t_truth / n_eval, results=rows,
                seconds=time.perf_counter() - t0)


def quick(ctx=None, seed_eval: int = synth.BASE_SEED + 104, top_triples: int = 65536,
          budgets=(10 ** 6, 10 ** 7)) -> dict:
    """A short recall measurement for the benchmark: one held-out 200 x 2000
    dataset, its exhaustive order-5 top-100 (tensor path), and the 30-feature
    proposals of the heuristic and of a network trained briefly (two
    datasets, T = 256, one epoch) at each budget."""
    ctx = ctx or epi.Context(0)
    ds = make(ctx, seed_eval, False)
    t0 = time.perf_counter()
    truth = {tuple(int(x) for x in c) for c in epi.search(ds, 5, 100, path="tc").combs}
    t_ex = time.perf_counter() - t0
    train = [make(ctx, synth.BASE_SEED + 200 + i, i % 2 == 0) for i in range(2)]
    net = epi.MLP(ctx, 30, 256, seed=1)
    t1 = time.perf_counter()
    epi.proposer_train(net, train, 256, 1, 8192, 1e-3, 1e-4, 0.5, 7)
    t_train = time.perf_counter() - t1
    out = dict(metric="top-N recall at k=5 (recall@100 of the exhaustive order-5 top-100)", n_snps=200,
               n_samples=2000, features=30, top_triples=top_triples, exhaustive_seconds=t_ex,
               train_seconds=t_train, results=[])
    epi.proposer_search(ds, None, top_triples, 4096, 100, quad_features=True)   # order-4 table, warm-up
    for R in budgets:
        for name, scorer in (("heuristic", None), ("network", net)):
            t2 = time.perf_counter()
            r, st = epi.proposer_search(ds, scorer, top_triples, R, 100, quad_features=True)
            secs = time.perf_counter() - t2
            rec = len({tuple(int(x) for x in c) for c in r.combs} & truth) / 100.0
            out["results"].append(dict(ranking=name, budget=R, recall_at_100=rec, seconds=secs,
                                       exact_in_proposals=int(st["exact_in_proposals"])))
    net.close()
    for d in train + [ds]:
        d.close()
    return out


def evaluate_large(ctx=None, n_snps: int = 2000, n_samples: int = 4000, top_triples: int = 512,
                   train_triples: int = 256, budgets=(10 ** 6, 10 ** 7, 10 ** 8),
                   seed: int = synth.BASE_SEED + 5) -> dict:
    """The proposer at 2000 SNPs x 4000 samples, where the exhaustive order-5
    search (C(2000, 5) = 2.65e14 sets) is out of reach.

    Features are the 25 of orders 1-3 (the order-4 table, C(2000, 4) floats,
    does not fit; four-way scores computed per candidate would cost as much
    as scoring the candidate exactly).  The network is trained on a separate
    dataset of the same shape, every row of its T = train_triples candidate
    space labelled by its exact order-5 MI.  The evaluation dataset carries a
    planted 5-SNP parity.  Reference: the exact top-100 of the whole
    candidate space of T = top_triples (every candidate scored exactly).
    Reported: recall of that top-100 among the top-100 proposed by the
    network and by the heuristic at each budget, the proposals' exact scores,
    the ranking throughput, and where the planted set stands."""
    import numpy as np
    ctx = ctx or epi.Context(0)
    half = n_samples // 2
    dtrain = synth.make_dataset(n_snps, half, n_samples - half, seed=seed + 1000)
    dev = synth.make_dataset(n_snps, half, n_samples - half, seed=seed, plant_q=5, plant_e=0.25)
    train = epi.Dataset(ctx, dtrain.geno, dtrain.pheno)
    ds = epi.Dataset(ctx, dev.geno, dev.pheno)
    net = epi.MLP(ctx, 25, 256, seed=1)
    t0 = time.perf_counter()
    losses = epi.proposer_train(net, [train], train_triples, 2, 8192, 1e-3, 1e-4, 0.5, 7)
    t_train = time.perf_counter() - t0
    # reference: every candidate of the space scored exactly (budget = all)
    epi.proposer_search(ds, None, 16, 4096, 100)            # lower-order tables, warm-up
    t0 = time.perf_counter()
    ref, st_ref = epi.proposer_search(ds, None, top_triples, 1 << 30, 100)
    t_ref = time.perf_counter() - t0
    space = int(st_ref["kept"])
    assert int(st_ref["proposals"]) == space, "the reference must score every candidate"
    truth = {tuple(int(x) for x in c) for c in ref.combs[:100]}
    out = dict(n_snps=n_snps, n_samples=n_samples, features=25, top_triples=top_triples,
               candidates=int(st_ref["candidates"]), distinct_candidates=space,
               reference=dict(seconds=t_ref, best_mi=float(ref.mi[0]), mi_100th=float(ref.mi[99]),
                              exact_in_proposals=int(st_ref["exact_in_proposals"])),
               training=dict(dataset="2000 x 4000, no plant", top_triples=train_triples, epochs=2,
                             seconds=t_train, losses=[float(x) for x in losses]),
               results=[])
    for R in budgets:
        for name, scorer in (("heuristic", None), ("network", net)):
            epi.proposer_search(ds, scorer, top_triples, R, 100)
            t1 = time.perf_counter()
            r, st = epi.proposer_search(ds, scorer, top_triples, R, 100)
            secs = time.perf_counter() - t1
            got = {tuple(int(x) for x in c) for c in r.combs}
            out["results"].append(dict(ranking=name, budget=R, recall_at_100=len(got & truth) / 100.0,
                                       seconds=secs, ranked_per_s=st["candidates"] / (st["ms_rank"] / 1e3),
                                       best_mi=float(r.mi[0]), mi_100th=float(r.mi[-1]),
                                       exact_in_proposals=int(st["exact_in_proposals"])))
    # the planted set: its exact score and its place among the candidates
    pl = tuple(int(x) for x in dev.planted)
    t = epi.tables(ds, np.array([pl], dtype=np.uint32))
    _, mi64 = epi.score_tables(ds, 5, t)
    ref_list = [tuple(int(x) for x in c) for c in ref.combs]
    out["planted"] = dict(snps=list(pl), mi=float(mi64[0]),
                          rank_among_candidates=(ref_list.index(pl) + 1) if pl in ref_list else None,
                          in_candidate_space=pl in ref_list or float(mi64[0]) <= float(ref.mi[-1]),
                          note="a pure 5-way parity has no lower-order signal, so no lower-order screen "
                               "expands it; its MI exceeds every candidate's, so it would rank first "
                               "wherever it is in the candidate space")
    net.close()
    train.close()
    ds.close()
    return out


def search_once(ctx=None, top_triples: int = 65536, budget: int = 10 ** 7, seed_net: int = 1) -> dict:
    """One 30-feature proposer search at 200 SNPs x 2000 samples with an
    untrained network (throughput only; for launch lists and timing), after a
    warm-up search that builds the lower-order tables."""
    ctx = ctx or epi.Context(0)
    ds = make(ctx, synth.BASE_SEED + 104, False)
    net = epi.MLP(ctx, 30, 256, seed=seed_net)
    epi.proposer_search(ds, net, 256, 4096, 100)
    t0 = time.perf_counter()
    r, st = epi.proposer_search(ds, net, top_triples, budget, 100)
    secs = time.perf_counter() - t0
    net.close()
    ds.close()
    return dict(top_triples=top_triples, budget=budget, seconds=secs, candidates=int(st["candidates"]),
                kept=int(st["kept"]), ms_rank=st["ms_rank"], ms_rescore=st["ms_rescore"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--search-once", action="store_true",
                    help="only time one 30-feature search (untrained network, T = 65536, R = 10^7)")
    ap.add_argument("--train", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=4, help="epochs of the 25-feature network")
    ap.add_argument("--epochs30", type=int, default=2, help="epochs of the 30-feature network")
    ap.add_argument("--train-triples", type=int, default=1024)
    ap.add_argument("--eval", type=int, default=3)
    args = ap.parse_args()
    if args.search_once:
        print(json.dumps(search_once()), flush=True)
        return
    print(json.dumps(evaluate(n_train=args.train, epochs=args.epochs, epochs30=args.epochs30,
                              train_triples=args.train_triples, n_eval=args.eval)), flush=True)


if __name__ == "__main__":
    main()
