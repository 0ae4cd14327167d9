"""Train the schedule-selection MLP from the library's own measured timings.

For every training graph (the batch mix: ER, path, grid, R-MAT with
log-uniform n in [1e3, 1e6]):
  1. compute its 12 features on the GPU (cc_batch_features);
  2. time all 18 schedules (order {2, 4, full chain} x {sync, async} x check
     interval {1, 2, 4}) with cc_run, taking the faster of two device-timed
     runs each; every schedule returns identical labels;
  3. label the graph with its fastest schedule; when several schedules are
     within 3% of the fastest, the one with the smallest median time (relative
     to each graph's best) over all training graphs is taken, so that
     near-ties do not turn measurement noise into label noise.
Then train the MLP on the GPU (cc_sched_train) and write the weight blob.

A second model serves batched solves (cc_sched_load_batch).  Inside a batch
a round lasts as long as its slowest graph and every graph is checked after
every sweep, so a graph's share of the batch is its sweep count times what
a sweep of its edges costs with the chosen order.  Its label is the
asynchronous order (2, 4 or the full chain) minimising that product: sweeps
as measured in a batched solve of the graph's chunk (after cc_batch_reorder,
as batched solves run), cost per swept edge from the same batches' device
times.

Held-out evaluation: graphs drawn from another seed plus large R-MAT (up to
scale 25), grid, path and caterpillar graphs; each is solved with
  plain    order 2, synchronous, c = 1 (the library's fallback schedule),
  C-2      order 2, asynchronous, c = 1 (the paper's default variant),
  learned  CC_ORDER_AUTO (feature extraction and inference included),
and the learned labels are checked to equal the plain ones.

Usage: python -m paper_2311_02811_gb300.sched_train [--train 20000]
       [--heldout 512] [--out paper_2311_02811_gb300/sched_weights.bin]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import graphgen as gg  # noqa: E402
import paper_2311_02811_gb300 as cc  # noqa: E402

TRAIN_SEED = 2311028110 + 50
HELDOUT_SEED = 2311028110 + 51


def time_schedules(n, s, d, reps=2):
    """Device solve time (ms) of each of the 18 schedules; the labels of all
    schedules are compared with each other."""
    g = cc.cc_init(n, s, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    ref = None
    times = np.zeros(cc.CC_SCHED_CLASSES)
    for k in range(cc.CC_SCHED_CLASSES):
        order, mode, c = cc.cc_sched_decode(k)
        best = float("inf")
        for _ in range(reps):
            st = cc.cc_run(g, out, order, mode, c)
            best = min(best, st.solve_ms)
        times[k] = best
        if ref is None:
            ref = out.clone()
        elif not torch.equal(ref, out):
            raise RuntimeError("schedules disagree on the labels")
    cc.cc_free(g)
    return times


# the classes a batch can use: order 2, 4 or the full chain, asynchronous
# (a batch checks every graph after every sweep)
BATCH_CLASSES = (3, 9, 15)


def batch_runs(plan, out):
    """Each BATCH_CLASSES schedule on a plan: the sweeps of every graph (G x 3)
    and the batch's device time per solve (3,), the faster of two runs."""
    cols, ms = [], []
    for k in BATCH_CLASSES:
        order, mode, c = cc.cc_sched_decode(k)
        cc.cc_batch_run(plan, out, order, mode, c)
        sw, t = cc.cc_batch_run(plan, out, order, mode, c)
        cols.append(np.asarray(sw))
        ms.append(t)
    return np.stack(cols, axis=1), np.array(ms)


def build_batch_set(n_graphs, chunk, log):
    """Features (after cc_batch_reorder, as batched solves run) and, for every
    graph, the sweeps it took in a batched solve of its chunk with each
    BATCH_CLASSES schedule; per chunk, the batch time of each schedule and
    the sum over its graphs of sweeps x edges."""
    feats, sweeps, ms_all, swm_all = [], [], [], []
    done = 0
    while done < n_graphs:
        cnt = min(chunk, n_graphs - done)
        vo, eo, s, d, _ = gg.batch_mix(cnt, seed=gg.stream_key(TRAIN_SEED, done), device="cuda")
        plan = cc.cc_batch_init(vo, eo, s, d)
        cc.cc_batch_reorder(plan)
        feats.append(cc.cc_batch_features(plan))
        out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
        sw, ms = batch_runs(plan, out)
        cc.cc_batch_free(plan)
        m = np.diff(eo).astype(np.float64)
        sweeps.append(sw)
        ms_all.append(ms)
        swm_all.append((sw * m[:, None]).sum(axis=0))
        done += cnt
        del s, d, out
        torch.cuda.empty_cache()
    log(f"batch training graphs: {done}")
    return (np.concatenate(feats).astype(np.float32), np.concatenate(sweeps), np.array(ms_all),
            np.array(swm_all))


def label_batch(Sw, ms, swm):
    """Batch label: the schedule with which the graph took the fewest sweeps
    in its batched solve (a round lasts as long as its slowest graph); at
    equal sweeps, the schedule whose training batches ran fastest overall.
    A cost-per-swept-edge label was tried and lost on held-out batches: a
    wrongly cheaper order that needs one more sweep lengthens its whole wave,
    which costs more than a cheaper sweep saves."""
    total = ms.sum(axis=0)
    rank = np.argsort(np.argsort(total))  # 0 = fastest over the training batches
    key = Sw * len(BATCH_CLASSES) + rank[None, :]
    return np.array(BATCH_CLASSES)[np.argmin(key, axis=1)].astype(np.int32), total / swm.sum(axis=0)


def build_training_set(n_graphs, chunk, log):
    feats, all_times = [], []
    done = 0
    while done < n_graphs:
        cnt = min(chunk, n_graphs - done)
        vo, eo, s, d, _ = gg.batch_mix(cnt, seed=gg.stream_key(TRAIN_SEED, done), device="cuda")
        plan = cc.cc_batch_init(vo, eo, s, d)
        F = cc.cc_batch_features(plan)
        cc.cc_batch_free(plan)
        for g in range(cnt):
            a, b = int(eo[g]), int(eo[g + 1])
            t = time_schedules(int(vo[g + 1] - vo[g]), s[a:b], d[a:b])
            feats.append(F[g])
            all_times.append(t)
        done += cnt
        del s, d
        torch.cuda.empty_cache()
        log(f"training graphs: {done}/{n_graphs}")
    T = np.array(all_times)
    return np.array(feats, np.float32), label_times(T), T


def train_batch_model(args, log):
    """The batch model: trained on label_batch labels; returns (blob, report)."""
    Xb, Sw, ms, swm = build_batch_set(args.train, args.chunk, log)
    yb, cost = label_batch(Sw, ms, swm)
    idx = np.arange(len(yb))
    val = idx % 10 == 0
    blob_b, loss_b = cc.cc_sched_train(Xb[~val], yb[~val], epochs=args.epochs, batch=256, lr=2e-3, seed=8)
    cc.cc_sched_load_batch(blob_b)
    pred_b, _ = cc.cc_sched_predict_batch(Xb[val])
    val_acc_b = float((pred_b == yb[val]).mean())
    col = {k: i for i, k in enumerate(BATCH_CLASSES)}
    key = Sw[val] * cost[None, :]
    chosen = key[np.arange(val.sum()), [col.get(int(k), 2) for k in pred_b]]
    cost_ratio_b = float(chosen.sum() / key.min(axis=1).sum())
    blob_b, loss_b = cc.cc_sched_train(Xb, yb, epochs=args.epochs, batch=256, lr=2e-3, seed=8)
    cc.cc_sched_load_batch(blob_b)
    with open(args.out_batch, "wb") as f:
        f.write(blob_b)
    log(f"batch model: loss {loss_b:.4f}, validation accuracy {val_acc_b:.3f}, est. cost vs best {cost_ratio_b:.3f}")
    return {"label_histogram": np.bincount(yb, minlength=cc.CC_SCHED_CLASSES).tolist(),
            "cost_per_swept_edge_ms": cost.tolist(), "final_loss": loss_b,
            "validation_accuracy": val_acc_b, "validation_est_cost_ratio_to_best": cost_ratio_b}


def evaluate_batch(n_mix, log, reps=3):
    """The held-out mix as one batch (reordered): each fixed batch schedule
    and the learned per-graph schedule, device time per solve."""
    vo, eo, s, d, _ = gg.batch_mix(n_mix, seed=HELDOUT_SEED, device="cuda")
    plan = cc.cc_batch_init(vo, eo, s, d, autotune=1)
    cc.cc_batch_reorder(plan)
    out = torch.empty(int(vo[-1]), dtype=torch.int32, device="cuda")
    res = {}
    ref = None
    for name, (order, mode, c) in (("batched-c2", (2, cc.CC_ASYNC, 1)), ("batched-o4", (4, cc.CC_ASYNC, 1)),
                                   ("batched-full", (cc.CC_ORDER_FULL, cc.CC_ASYNC, 1)),
                                   ("batched-plain", (2, cc.CC_SYNC, 1)),
                                   ("batched-learned", (cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0))):
        cc.cc_batch_run(plan, out, order, mode, c)
        res[name] = min(cc.cc_batch_run(plan, out, order, mode, c)[1] for _ in range(reps))
        if ref is None:
            ref = out.clone()
        elif not torch.equal(ref, out):
            raise RuntimeError("batched schedules disagree on the labels")
    cc.cc_batch_free(plan)
    log(f"held-out batch ({n_mix} graphs): {res}")
    return res


def label_times(T, tol=1.03):
    """Fastest schedule per row; near-ties broken by the global median ratio."""
    ratio = T / T.min(axis=1, keepdims=True)
    pref = np.argsort(np.argsort(np.median(ratio, axis=0)))  # rank of each schedule
    near = ratio <= tol
    score = np.where(near, pref[None, :], len(pref) + 1)
    return np.argmin(score, axis=1).astype(np.int32)


def heldout_graphs(n_mix):
    """(name, n, src, dst) of the held-out set, generated one at a time."""
    params = gg.batch_mix_params(n_mix, seed=HELDOUT_SEED)
    for i, p in enumerate(params):
        n, s, d = gg.batch_graph(p, device="cuda")
        yield f"mix{i}-{p['kind']}", n, s, d
    for scale in (20, 22, 24, 25):
        s, d = gg.rmat(scale, seed=HELDOUT_SEED + scale, device="cuda")
        yield f"rmat{scale}", 1 << scale, s, d
    for side in (1024, 2048, 4096):
        s, d = gg.grid(side, side, seed=HELDOUT_SEED + side, device="cuda")
        yield f"grid{side}", side * side, s, d
    for n in (1 << 20, 1 << 23):
        s, d = gg.path(n, seed=HELDOUT_SEED + 7, device="cuda")
        yield f"path{n}", n, s, d
    s, d = gg.caterpillar(1 << 20, seed=HELDOUT_SEED + 8, device="cuda")
    yield "caterpillar2^20", (1 << 20) * 16, s, d


def evaluate(n_mix, log):
    """Each form on a fresh handle: the first call (cold: loop-graph build and,
    for the learned form, features and inference) and the best of 3 later calls."""
    rows = []
    stream = torch.cuda.current_stream()

    def ev_time(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    for name, n, s, d in heldout_graphs(n_mix):
        row = {"graph": name, "n": n, "m": int(s.numel())}
        outs = {}
        for form, (order, mode, c) in (("plain", (2, cc.CC_SYNC, 1)), ("c2", (2, cc.CC_ASYNC, 1)),
                                       ("learned", (cc.CC_ORDER_AUTO, cc.CC_ASYNC, 0))):
            g = cc.cc_init(n, s, d)
            out = torch.empty(n, dtype=torch.int32, device="cuda")
            first, st = ev_time(lambda: cc.cc_run(g, out, order, mode, c))
            steady = min(ev_time(lambda: cc.cc_run(g, out, order, mode, c))[0] for _ in range(3))
            cc.cc_free(g)
            row[f"{form}_first_ms"] = first
            row[f"{form}_ms"] = steady
            if form == "learned":
                row["learned_schedule"] = [st.order, st.mode, st.check_interval]
            outs[form] = out
        row["identical"] = bool(torch.equal(outs["plain"], outs["learned"]) and torch.equal(outs["plain"], outs["c2"]))
        rows.append(row)
        del s, d, outs
        torch.cuda.empty_cache()
    keys = ("plain_ms", "c2_ms", "learned_ms", "plain_first_ms", "c2_first_ms", "learned_first_ms")
    tot = {k: sum(r[k] for r in rows) for k in keys}
    log(f"held-out totals: {tot}")
    return rows, tot


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=496, help="batch-mix graphs; 16 large graphs are added")
    ap.add_argument("--chunk", type=int, default=500)
    ap.add_argument("--epochs", type=int, default=80)
    ap.add_argument("--out", default=os.path.join(HERE, "sched_weights.bin"))
    ap.add_argument("--out-batch", default=os.path.join(HERE, "sched_weights_batch.bin"))
    ap.add_argument("--report", default=os.path.join(os.path.dirname(HERE), "profiles", "sched_weights.json"))
    ap.add_argument("--dump", default="", help="also save features, labels and timings (.npz)")
    ap.add_argument("--batch-only", action="store_true",
                    help="train only the batch model (the single-graph weights in --out stay)")
    ap.add_argument("--eval-only", action="store_true",
                    help="evaluate the weights in --out on the held-out set and update the report")
    args = ap.parse_args()
    t0 = time.time()

    def log(msg):
        print(f"[{time.time() - t0:7.1f}s] {msg}", flush=True)

    torch.cuda.set_device(0)
    if args.eval_only:
        cc.load_default_scheduler(args.out, args.out_batch)
        batch_eval = evaluate_batch(args.heldout, log)
        rows, tot = evaluate(args.heldout, log)
        report = json.load(open(args.report)) if os.path.exists(args.report) else {}
        report.update({"heldout_totals_ms": tot,
                       "heldout_speedup_vs_plain": tot["plain_ms"] / tot["learned_ms"],
                       "heldout_speedup_vs_c2": tot["c2_ms"] / tot["learned_ms"],
                       "heldout_first_call_speedup_vs_plain": tot["plain_first_ms"] / tot["learned_first_ms"],
                       "heldout_first_call_speedup_vs_c2": tot["c2_first_ms"] / tot["learned_first_ms"],
                       "heldout_all_identical": all(r["identical"] for r in rows), "heldout": rows})
        report.setdefault("batch_model", {})["heldout_batch_ms"] = batch_eval
        with open(args.report, "w") as f:
            json.dump(report, f, indent=0, separators=(",", ":"))
        log(f"updated {args.report}")
        return
    if args.batch_only:
        cc.load_default_scheduler(args.out, None)
        report = json.load(open(args.report)) if os.path.exists(args.report) else {}
        bm = train_batch_model(args, log)
        bm["heldout_batch_ms"] = evaluate_batch(args.heldout, log)
        report["batch_model"] = bm
        with open(args.report, "w") as f:
            json.dump(report, f, indent=0, separators=(",", ":"))
        log(f"wrote {args.out_batch} and {args.report}")
        return
    X, y, T = build_training_set(args.train, args.chunk, log)
    if args.dump:
        np.savez_compressed(args.dump, X=X, y=y, T=T)
    # 90/10 split for a validation accuracy; the final model trains on all rows
    idx = np.arange(len(y))
    val = idx % 10 == 0
    blob, loss = cc.cc_sched_train(X[~val], y[~val], epochs=args.epochs, batch=256, lr=2e-3, seed=7)
    cc.cc_sched_load(blob)
    pred, _ = cc.cc_sched_predict(X[val])
    val_acc = float((pred == y[val]).mean())
    # time of the predicted schedule relative to the best one, on validation rows
    regret = float(np.mean(T[val][np.arange(val.sum()), pred] / T[val].min(axis=1)))
    blob, loss = cc.cc_sched_train(X, y, epochs=args.epochs, batch=256, lr=2e-3, seed=7)
    cc.cc_sched_load(blob)
    log(f"trained: loss {loss:.4f}, validation accuracy {val_acc:.3f}, mean time ratio to best {regret:.3f}")
    with open(args.out, "wb") as f:
        f.write(blob)
    bm = train_batch_model(args, log)
    bm["heldout_batch_ms"] = evaluate_batch(args.heldout, log)
    rows, tot = evaluate(args.heldout, log)
    label_hist = np.bincount(y, minlength=cc.CC_SCHED_CLASSES).tolist()
    report = {"train_graphs": int(len(y)), "label_histogram": label_hist, "final_loss": loss,
              "validation_accuracy": val_acc, "validation_time_ratio_to_best": regret,
              "heldout_totals_ms": tot,
              "heldout_speedup_vs_plain": tot["plain_ms"] / tot["learned_ms"],
              "heldout_speedup_vs_c2": tot["c2_ms"] / tot["learned_ms"],
              "heldout_first_call_speedup_vs_plain": tot["plain_first_ms"] / tot["learned_first_ms"],
              "heldout_first_call_speedup_vs_c2": tot["c2_first_ms"] / tot["learned_first_ms"],
              "heldout_all_identical": all(r["identical"] for r in rows),
              "batch_model": bm,
              "heldout": rows}
    with open(args.report, "w") as f:
        json.dump(report, f, indent=0, separators=(",", ":"))
    log(f"wrote {args.out}, {args.out_batch} and {args.report}")


if __name__ == "__main__":
    main()
