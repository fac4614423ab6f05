"""Learned parameter predictor: data from the grid search, training on the
GPU, regret against the grid search.

Section 5 of the paper caches optimizer timings of small squares and
rectangles of sizes 2^a 3^b 5^c 7^d and fits classifiers to them (Section
5.3: classification beats regression); Section 4.2 searches each axis on its
own.  Here:

* ``collect``: 2-D squares and rectangles with sides in the 2^a 3^b 5^c 7^d
  sizes of [16, 512] (plus skinny rectangles of height 4 to 32), each
  searched by the exhaustive tuner (``hdc_tune_convnd``) on the GPU; the
  record keeps the best (m, p, q, D) per axis and its time.
* ``samples``: one sample per axis: the HDC_MLP_FEATURES features of the
  axis in its problem, the class of its best residue count q and whether
  its best D was q (all residues in one pass) or less.
* ``train``: full-batch Adam on the GPU with the library's forward,
  backward and Adam kernels; the initial weights are drawn on the host.
* ``evaluate``: for larger problems (2-D rectangles up to 4096 x 2048, 3-D
  cubes up to 256^3) the regret T(predicted) / T(grid-search best) - 1 of
  the top class per axis, and of a search over the predictor's three best
  classes per axis (about 3 timed runs per axis instead of the grid's
  dozens), beside two predictor-free rules: explicit padding (q = 1 per
  axis) and a fixed q = 2 per axis.

    python -m paper_2306_10016_gb300.predictor --out DIR [--collect N]
           [--train STEPS] [--eval] [--dataset FILE] [--weights FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import synth


def good_sizes(lo: int, hi: int):
    out = []
    for n in range(lo, hi + 1):
        k = n
        for f in (2, 3, 5, 7):
            while k % f == 0:
                k //= f
        if k == 1:
            out.append(n)
    return out


def training_problems(seed: int, n_rect: int):
    """All squares with sides in the 7-smooth sizes of [16, 512], skinny
    rectangles of heights 4..32, n_rect seeded rectangles, and rectangles of
    height 16 and 32 whose long side runs through the 7-smooth sizes of
    (512, 4096]: every training problem holds at most 512 x 512 outputs, but
    axes as long as those of the larger problems the predictor is used on
    appear in them (the paper's transfer from rectangles to squares,
    Section 5.3 and Section 6.2)."""
    sides = good_sizes(16, 512)
    probs = [(s, s) for s in sides]
    for s in sides[::3]:
        for h in (4, 8, 16, 32):
            probs.append((s, h))
            probs.append((h, s))
    for s in good_sizes(513, 4096)[::2]:
        for h in (16, 32):
            if s * h <= 512 * 512:
                probs.append((s, h))
                probs.append((h, s))
    u = synth.uniform01(seed, 2 * n_rect)
    for k in range(n_rect):
        a = sides[int(u[2 * k] * len(sides))]
        b = sides[int(u[2 * k + 1] * len(sides))]
        probs.append((a, b))
    seen, out = set(), []
    for p in probs:
        if p not in seen:
            seen.add(p)
            out.append(p)
    return out


def collect(problems, dtype=None, max_ratio=1.5, reps=3, log=None):
    import torch

    import paper_2306_10016_gb300 as hdc
    dtype = hdc.HDC_C128 if dtype is None else dtype
    tdt = torch.complex128 if dtype == hdc.HDC_C128 else torch.complex64
    recs = []
    for k, shape in enumerate(problems):
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 50 + k, shape)).to("cuda", tdt)
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 5050 + k, shape)).to("cuda", tdt)
        best, trials = hdc.tune(f, g, len(shape), max_ratio=max_ratio, reps=reps)
        recs.append({"L": list(shape), "M": [2 * x - 1 for x in shape], "dtype": int(dtype), "batch": 1,
                     "best": [{k2: b[k2] for k2 in ("m", "p", "q", "D")} for b in best],
                     "ms": best[0]["ms"],
                     "trials": [[[t["m"], t["q"], t["D"]] for t in tr] + [tr[0]["ms"]] for tr in trials]})
        if log and k % 20 == 0:
            log(f"collect {k}/{len(problems)} {shape} -> {recs[-1]['best']}")
    return recs


def axis_label(rec, axis, tol=0.03):
    """(q, D) label of one axis: among the configurations of that axis'
    sweep (the trials in which only this axis varies) that run within
    `tol` of the fastest, the one with the fewest residues -- timings of
    small problems tie often, and fewer residues carry over to larger ones."""
    trials = rec.get("trials")
    best = rec["best"][axis]
    if not trials or isinstance(trials, int):
        return best["q"], best["D"]
    groups = {}
    for tr in trials:
        cfg, ms = tr[:-1], tr[-1]
        key = tuple(tuple(c) for a, c in enumerate(cfg) if a != axis)
        groups.setdefault(key, []).append((cfg[axis], ms))
    sweep = max(groups.values(), key=len)
    fastest = min(ms for _, ms in sweep)
    ok = [c for c, ms in sweep if ms <= (1.0 + tol) * fastest]
    m, q, D = min(ok, key=lambda c: (c[1], -c[2], c[0]))
    return q, D


def samples(records, tol=0.03):
    import paper_2306_10016_gb300 as hdc
    X, yq, yd = [], [], []
    for r in records:
        feats = hdc.mlp_axis_features(r["L"], r["M"], r["dtype"], r.get("batch", 1))
        for a in range(len(r["L"])):
            q, D = axis_label(r, a, tol)
            X.append(feats[a])
            yq.append(hdc.mlp_q_to_class(q))
            yd.append(0 if D >= q else 1)
    return (np.array(X, dtype=np.float32), np.array(yq, dtype=np.int32), np.array(yd, dtype=np.int32))


def init_params(n_in, hidden, n_out, seed):
    """Uniform weights in +-sqrt(6 / fan_in) (He et al., 2015), zero biases."""
    dims = [n_in, hidden, hidden, hidden, n_out]
    parts = []
    for l in range(4):
        nw = dims[l] * dims[l + 1]
        bound = math.sqrt(6.0 / dims[l])
        parts.append((2.0 * synth.uniform01(seed + l, nw) - 1.0) * bound)
        parts.append(np.zeros(dims[l + 1]))
    return np.concatenate(parts).astype(np.float32)


def train(X, yq, yd, steps=3000, lr=3e-3, seed=230610016, log=None, checkpoint=None, resume=None):
    """Full-batch Adam on the GPU; returns (network, loss history)."""
    import torch

    import paper_2306_10016_gb300 as hdc
    net = hdc.MLP(n_in=X.shape[1])
    if resume and os.path.exists(resume):
        net.load(resume)
    else:
        net.set_params(init_params(net.n_in, net.hidden, net.n_out, seed))
    Xd = torch.from_numpy(X).cuda()
    yqd = torch.from_numpy(yq).cuda()
    ydd = torch.from_numpy(yd).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for it in range(steps):
        net.loss_grad(Xd, yqd, ydd, loss)
        net.adam(lr)
        if it % 100 == 0 or it == steps - 1:
            hist.append((it, float(loss.item())))
            if log:
                log(f"train step {it} loss {hist[-1][1]:.4f}")
    if checkpoint:
        net.save(checkpoint)
    return net, hist


def accuracy(net_or_params, X, yq, yd):
    """Classification accuracy of both heads (q class, D class)."""
    import torch
    logits = net_or_params.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    nq = logits.shape[1] - 2
    aq = float(np.mean(np.argmax(logits[:, :nq], axis=1) == yq))
    ad = float(np.mean(np.argmax(logits[:, nq:], axis=1) == yd))
    return aq, ad


def _time_params(f, g, dims, prm, reps=5):
    import torch

    import paper_2306_10016_gb300 as hdc
    m = [p["m"] for p in prm]
    D = [p["D"] for p in prm]
    L = list(f.shape[-dims:])
    ws = torch.empty(hdc.workspace_size(L, [2 * x - 1 for x in L], m, D=D), dtype=torch.uint8, device=f.device)
    h = torch.empty_like(f)
    for _ in range(2):
        hdc.convnd(f, g, dims, m, D=D, out=h, workspace=ws)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        hdc.convnd(f, g, dims, m, D=D, out=h, workspace=ws)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _rule_params(L, q, dtype=None):
    """q residues per axis (more on an outer axis whose m would exceed the
    column-tile limit)."""
    import paper_2306_10016_gb300 as hdc
    dtype = hdc.HDC_C128 if dtype is None else dtype
    out = []
    for a, l in enumerate(L):
        M = 2 * l - 1
        qa = q
        while True:
            m = hdc.next_good_size(-(-M // qa))
            if a == len(L) - 1 or m <= hdc.max_outer_fft_size(dtype):
                break
            qa += 1
        rc, (p, qq, D) = hdc.validate_axis(l, M, m, dtype=dtype)
        out.append(dict(m=m, p=p, q=qq, D=D))
    return out


# seed and count of the seeded training rectangles (the packaged dataset's)
TRAIN_SEED = synth.BASE_SEED + 5
TRAIN_RECTANGLES = 240

EVAL_PROBLEMS = [(768, 768), (1024, 1024), (2048, 512), (2048, 1024), (3072, 1536), (4096, 2048),
                 (32, 32, 32), (64, 64, 64), (128, 128, 128), (256, 256, 256)]


KEYS = ("mlp", "mlp_top3", "random25", "proxy32", "explicit", "q2")


def evaluate(weights, problems=None, dtype=None, reps=5, log=None):
    import torch

    import paper_2306_10016_gb300 as hdc
    dtype = hdc.HDC_C128 if dtype is None else dtype
    tdt = torch.complex128 if dtype == hdc.HDC_C128 else torch.complex64
    rows = []
    for k, shape in enumerate(problems or EVAL_PROBLEMS):
        dims = len(shape)
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 90 + k, shape)).to("cuda", tdt)
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 9090 + k, shape)).to("cuda", tdt)
        t0 = time.perf_counter()
        best, search_trials = hdc.tune(f, g, dims, max_ratio=1.5, reps=3)
        t_search = time.perf_counter() - t0
        # the paper's cheap searches (Section 4.3 random search, Section 6.3
        # height-32 rectangle) as baselines for the predictor
        t0 = time.perf_counter()
        rbest, rtrials = hdc.tune_random(f, g, dims, max_ratio=1.5, reps=3)
        t_random = time.perf_counter() - t0
        t0 = time.perf_counter()
        xbest, xtimed = hdc.tune_proxy(f, g, dims, 32, max_ratio=1.5, reps=3)
        t_proxy = time.perf_counter() - t0
        t0 = time.perf_counter()
        pred = hdc.Plan(list(shape), dtype=dtype, mode=hdc.HDC_PREDICT_MLP, tuning_db=str(weights)).params
        t_pred = time.perf_counter() - t0
        t0 = time.perf_counter()
        gplan = hdc.Plan(list(shape), dtype=dtype, mode=hdc.HDC_PREDICT_MLP_SEARCH, tuning_db=str(weights))
        guided, n_timed = gplan.params, gplan.timed
        t_guided = time.perf_counter() - t0
        def prm(bs):
            return [dict(m=b["m"], p=b["p"], q=b["q"], D=b["D"]) for b in bs]

        cand = {"search": prm(best), "mlp": pred, "mlp_top3": guided, "random25": prm(rbest), "proxy32": prm(xbest),
                "explicit": _rule_params(shape, 1, dtype), "q2": _rule_params(shape, 2, dtype)}
        t = {k2: _time_params(f, g, dims, v, reps) for k2, v in cand.items()}
        row = {"shape": list(shape), "ms": {k2: round(v, 4) for k2, v in t.items()},
               "regret": {k2: round(t[k2] / t["search"] - 1.0, 4) for k2 in KEYS},
               "params": cand, "search_s": round(t_search, 2), "search_timed": len(search_trials),
               "predict_s": round(t_pred, 4), "top3_s": round(t_guided, 2), "top3_timed": n_timed,
               "random_s": round(t_random, 2), "random_timed": len(rtrials), "proxy_s": round(t_proxy, 2),
               "proxy_timed": int(xtimed)}
        rows.append(row)
        if log:
            log(f"eval {shape}: {row['ms']} regret {row['regret']}")
        del f, g
        torch.cuda.empty_cache()

    def stats(key):
        r = np.array([max(0.0, x["regret"][key]) for x in rows])
        return {"geomean": float(np.exp(np.mean(np.log1p(r))) - 1.0), "p90": float(np.quantile(r, 0.9)),
                "max": float(r.max())}

    return {"rows": rows, "summary": {k2: stats(k2) for k2 in KEYS}}


# ------------------------------------------------ held-out timing records
# The predictor's top class is judged on problems larger than any it was
# trained on, by device times measured once on the GPU and kept with the
# package: per problem the grid search's choice and time, and the time of
# every combination of per-axis choices m = nextgood(ceil(M / q_k)) with
# D = q (and D = 1 in 2-D) over the residue-count classes q_k (q_k <= 4 in
# 3-D), plus the packaged network's own choice.  Regret of any choice in
# the table is then computed on the host.

def _graph_ms(run, reps=5):
    """Median device time (ms) of run(stream) replayed from a CUDA graph, L2
    evicted before each replay (as the tuner and the throughput measurement
    time)."""
    import torch
    flush = _graph_ms.flush
    if flush is None:
        flush = _graph_ms.flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        run(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        run(side)
    graph.replay()
    st = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        graph.replay()
        e1.record(st)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    del graph
    return float(np.median([a.elapsed_time(b) for a, b in ts]))


_graph_ms.flush = None


def combo_key(prm):
    return "|".join(f"{p['m']}:{p['D']}" for p in prm)


def axis_options(L, dims, a, dtype, with_one):
    """The (m, p, q, D) one axis can take from the q classes (deduplicated
    by (m, D)); D = q, and D = 1 too when with_one."""
    import ctypes

    import paper_2306_10016_gb300 as hdc
    M = 2 * L - 1
    max_m = hdc.max_outer_fft_size(dtype) if a < dims - 1 else 0
    out, seen = [], set()
    for k, qk in enumerate(hdc.mlp_q_classes()):
        if dims == 3 and qk > 4:
            continue
        for one in ((0, 1) if with_one else (0,)):
            v = [ctypes.c_int64() for _ in range(4)]
            rc = hdc.lib().hdc_mlp_decode_class(k, one, L, M, dtype, max_m, *[ctypes.byref(x) for x in v])
            if rc != 0:
                continue
            m, p, q, D = (x.value for x in v)
            if (m, D) not in seen:
                seen.add((m, D))
                out.append(dict(m=m, p=p, q=q, D=D))
    return out


def top_class_params(shape, dtype, logits_fn):
    """The network's most likely valid choice per axis (what HDC_PREDICT_MLP
    plans), from logits_fn(X) -> logits of the axes' features."""
    import paper_2306_10016_gb300 as hdc
    dims = len(shape)
    X = hdc.mlp_axis_features(list(shape), [2 * x - 1 for x in shape], dtype)
    lg = logits_fn(X)
    out = []
    for a, L in enumerate(shape):
        max_m = hdc.max_outer_fft_size(dtype) if a < dims - 1 else 0
        out.append(hdc.mlp_decode_axis(lg[a], L, 2 * L - 1, dtype, max_m))
    return out


def timing_records(weights, problems=None, dtype=None, reps=5, log=None):
    import itertools

    import torch

    import paper_2306_10016_gb300 as hdc
    dtype = hdc.HDC_C128 if dtype is None else dtype
    tdt = torch.complex128 if dtype == hdc.HDC_C128 else torch.complex64
    recs = []
    for k, shape in enumerate(problems or EVAL_PROBLEMS):
        dims = len(shape)
        f = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 90 + k, shape)).to("cuda", tdt)
        g = torch.from_numpy(synth.unit_disk(synth.BASE_SEED + 9090 + k, shape)).to("cuda", tdt)
        h = torch.empty_like(f)
        L = list(shape)
        Mv = [2 * x - 1 for x in L]

        def t_of(prm):
            m = [p["m"] for p in prm]
            D = [p["D"] for p in prm]
            ws = torch.empty(max(1, hdc.workspace_size(L, Mv, m, D=D, dtype=dtype)), dtype=torch.uint8,
                             device="cuda")
            return _graph_ms(lambda s_: hdc.convnd(f, g, dims, m, D=D, out=h, workspace=ws, stream=s_), reps)

        t0 = time.perf_counter()
        best, trials = hdc.tune(f, g, dims, max_ratio=1.5, reps=reps)
        t_search = time.perf_counter() - t0
        search = [dict(m=b["m"], p=b["p"], q=b["q"], D=b["D"]) for b in best]
        opts = [axis_options(x, dims, a, dtype, dims < 3) for a, x in enumerate(L)]
        table = {}
        configs = [list(c) for c in itertools.product(*opts)]
        net = hdc.Plan(L, dtype=dtype, mode=hdc.HDC_PREDICT_MLP, tuning_db=str(weights)).params if weights else None
        extra = [search, _rule_params(shape, 1, dtype), _rule_params(shape, 2, dtype)] + ([net] if net else [])
        for prm in configs + extra:
            key = combo_key(prm)
            if key not in table:
                table[key] = round(t_of(prm), 5)
        rec = {"shape": L, "dtype": int(dtype), "search": search, "search_ms": table[combo_key(search)],
               "search_s": round(t_search, 2), "search_timed": len(trials),
               "explicit": combo_key(_rule_params(shape, 1, dtype)), "q2": combo_key(_rule_params(shape, 2, dtype)),
               "network": combo_key(net) if net else None, "ms": table}
        recs.append(rec)
        if log:
            log(f"records {shape}: {len(table)} configurations, search {rec['search_ms']} ms")
        del f, g, h
        torch.cuda.empty_cache()
    return recs


def regret_table(records, choose):
    """Regret T(choice) / T(grid search) - 1 (clamped at 0) per record, for
    choose(record) -> configuration key (or None when not in the table), and
    the geometric mean, 90th percentile and maximum."""
    r = []
    for rec in records:
        key = choose(rec)
        if key is None or key not in rec["ms"]:
            r.append(float("nan"))
            continue
        best = min(rec["search_ms"], min(rec["ms"].values()))
        r.append(max(0.0, rec["ms"][key] / rec["search_ms"] - 1.0) if best > 0 else float("nan"))
    a = np.array(r)
    ok = a[np.isfinite(a)]
    return {"per_problem": r, "geomean": float(np.exp(np.mean(np.log1p(ok))) - 1.0) if ok.size else None,
            "p90": float(np.quantile(ok, 0.9)) if ok.size else None, "max": float(ok.max()) if ok.size else None,
            "missing": int(a.size - ok.size)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--collect", type=int, default=0, help="seeded rectangles beyond the squares (0: skip)")
    ap.add_argument("--dataset", default=None)
    ap.add_argument("--train", type=int, default=0)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--weights", default=None)
    ap.add_argument("--eval", action="store_true")
    ap.add_argument("--records", default=None, help="write held-out timing records (json.gz) of the weights")
    a = ap.parse_args(argv)
    os.makedirs(a.out, exist_ok=True)

    def log(msg):
        print(msg, flush=True)

    ds_path = a.dataset or os.path.join(a.out, "mlp_dataset.json")
    w_path = a.weights or os.path.join(a.out, "mlp_weights.bin")
    report = {}
    if a.collect:
        t0 = time.perf_counter()
        recs = collect(training_problems(TRAIN_SEED, a.collect), log=log)
        report["collect_s"] = round(time.perf_counter() - t0, 1)
        with open(ds_path, "w") as fh:
            json.dump(recs, fh)
    if a.train:
        with open(ds_path) as fh:
            recs = json.load(fh)
        X, yq, yd = samples(recs)
        t0 = time.perf_counter()
        net, hist = train(X, yq, yd, steps=a.train, lr=a.lr, log=log, checkpoint=w_path)
        report["train_s"] = round(time.perf_counter() - t0, 2)
        report["train_samples"] = int(X.shape[0])
        report["loss"] = hist
        aq, ad = accuracy(net, X, yq, yd)
        counts = np.bincount(yq, minlength=net.n_out - 2)
        report["train_accuracy"] = {"q": aq, "D": ad, "q_majority_rule": float(counts.max() / counts.sum())}
        log(f"train accuracy q {aq:.3f} D {ad:.3f} (majority {report['train_accuracy']['q_majority_rule']:.3f})")
    if a.records:
        t0 = time.perf_counter()
        recs = timing_records(w_path, log=log)
        report["records_s"] = round(time.perf_counter() - t0, 1)
        import gzip
        with gzip.open(a.records, "wt") as fh:
            json.dump(recs, fh)
        report["records_regret"] = {
            "network": regret_table(recs, lambda r: r["network"]),
            "explicit": regret_table(recs, lambda r: r["explicit"]),
            "q2": regret_table(recs, lambda r: r["q2"])}
        log(json.dumps(report["records_regret"]))
    if a.eval:
        report["eval"] = evaluate(w_path, log=log)
        log(json.dumps(report["eval"]["summary"]))
    with open(os.path.join(a.out, "mlp_report.json"), "w") as fh:
        json.dump(report, fh, indent=1)


if __name__ == "__main__":
    main()
