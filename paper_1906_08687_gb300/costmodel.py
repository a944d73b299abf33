"""Learned plan choice for the engine: timing corpus, training, regret.

The planner's candidates for a batch (lmf_plan_candidates: roots x Gram form)
are each planned, compiled and timed on the GPU; the cost
model (lmf_mlp, trained here with the engine's own forward/backward/Adam
kernels) learns log run time from the plan features; on held-out schemas its
choice is compared with the exhaustive best and with the paper's root rule
(Sec. 3.3), which stays the fallback.

    python -m paper_1906_08687_gb300.costmodel --schemas 500 --train 400 --scale 0.1
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import sys
import time
from typing import Dict, List, Optional

import numpy as np

from .lmf import (LMF_BATCH_GRAPH, LMF_PLAN_FEATURES, LMF_PLAN_NO_JIT, LMF_PREC_SPLIT_BF16, LMF_ROOT_HEURISTIC, Engine,
                  LmfError, Mlp, lmf_plan_opts, register_schema)


def _opts_tuple(o) -> tuple:
    return (o.precision, o.batching, o.tile_rows, o.ctas_per_sm, o.root_mode, o.root_rel, o.no_merge, o.flags)


def time_run(eng: Engine, bid: int, runs: int, max_ms: float) -> float:
    """Median CUDA-event time of `runs` runs after one warm-up (fewer when one
    run exceeds max_ms)."""
    import torch
    s = torch.cuda.Stream()
    eng.run(bid, s.cuda_stream)
    torch.cuda.synchronize()
    out = []
    for _ in range(runs):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        eng.run(bid, s.cuda_stream)
        b.record(s)
        torch.cuda.synchronize()
        out.append(a.elapsed_time(b))
        if out[-1] > max_ms:
            break
    eng.sync(bid)
    return float(statistics.median(out))


def collect(schemas, runs: int = 3, max_ms: float = 200.0, device: int = 0, log=None, jit: bool = True,
            threads: int = 16) -> List[Dict]:
    """schemas: iterable of (schema, batch).  One record per schema with every
    distinct candidate's features and time, and the root rule's plan and time.
    Candidates run the root scan compiled for their plan (the product path):
    the sources of all candidates of a schema are compiled first on `threads`
    host threads (lmf_plan_precompile), then each candidate is planned and
    timed.  Candidates that plan to the same thing (a key-level request that
    falls back to the row-level form, say) are timed once."""
    import torch
    recs = []
    for si, (sch, batch) in enumerate(schemas):
        tensors = {(r.name, c.name): torch.from_numpy(np.ascontiguousarray(c.data)).to(f'cuda:{device}')
                   for r in sch.relations for c in r.columns}
        eng = Engine(device)
        register_schema(eng, sch, tensors)
        bid = eng.declare_batch(batch)
        cands, feats, ms, seen = [], [], [], set()
        flags = 0 if jit else LMF_PLAN_NO_JIT
        base = lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, 0, 0, 0, flags)
        t0 = time.time()
        if jit:
            eng.plan_precompile(bid, base, threads)
        t_compile = time.time() - t0
        for o in eng.plan_candidates(bid, base):
            try:
                eng.plan_opts(bid, o)
            except LmfError:
                continue
            info = eng.plan_info(bid)
            key = (info['root_rel'], info['precision'], info['key_level'], o.no_merge)
            if key in seen:
                continue
            seen.add(key)
            feats.append(eng.plan_features(bid))
            ms.append(time_run(eng, bid, runs, max_ms))
            cands.append(_opts_tuple(o))
        h = lmf_plan_opts(LMF_PREC_SPLIT_BF16, LMF_BATCH_GRAPH, 0, 0, LMF_ROOT_HEURISTIC, 0, 0, flags)
        eng.plan_opts(bid, h)
        heur_ms = time_run(eng, bid, runs, max_ms)
        hi = eng.plan_info(bid)
        eng.close()
        del tensors
        best = int(np.argmin(ms))
        rec = {'name': sch.meta.get('name', str(si)), 'cand': cands, 'feat': np.array(feats, np.float32),
               'ms': np.array(ms, np.float64), 'heur_ms': heur_ms, 'heur_root': hi['root_rel'],
               'heur_key_level': hi['key_level'], 'n_aggs': len(batch), 'compile_s': t_compile,
               'rows': [r.nrows for r in sch.relations], 'best': cands[best]}
        recs.append(rec)
        if log:
            log(f'{si}: {rec["name"]} candidates={len(ms)} best={ms[best]:.3f}ms {cands[best]} '
                f'rule={heur_ms:.3f}ms root={hi["root_rel"]} rows={rec["rows"]} compile={t_compile:.1f}s')
    return recs


def fit_norm(X: np.ndarray, y: np.ndarray):
    mean = X.mean(axis=0)
    std = X.std(axis=0)
    std = np.where(std > 1e-6, std, 1.0)
    return mean.astype(np.float32), std.astype(np.float32), float(y.mean()), float(max(y.std(), 1e-6))


def train(recs: List[Dict], steps: int = 2000, lr: float = 1e-3, batch: int = 256, seed: int = 0,
          hidden: int = 128, device: int = 0):
    """Fit the cost model to log(ms) of every candidate of the given records."""
    import torch
    X = np.concatenate([r['feat'] for r in recs]).astype(np.float32)
    y = np.log(np.concatenate([r['ms'] for r in recs])).astype(np.float32)
    mean, std, ym, ys = fit_norm(X, y)
    model = Mlp(LMF_PLAN_FEATURES, hidden, seed, device)
    model.set_norm(mean, std, ym, ys)
    Xd = torch.from_numpy(X).to(f'cuda:{device}')
    yd = torch.from_numpy((y - ym) / ys).to(f'cuda:{device}')
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        idx = torch.from_numpy(rng.integers(0, len(X), size=min(batch, len(X)))).to(Xd.device)
        xb = Xd.index_select(0, idx).contiguous()
        yb = yd.index_select(0, idx).contiguous()
        losses.append(model.train_step(xb.data_ptr(), yb.data_ptr(), len(xb), lr))
    model.norm = (mean, std, ym, ys)
    return model, losses


def predict(model: Mlp, feats: np.ndarray, device: int = 0) -> np.ndarray:
    import torch
    x = torch.from_numpy(np.ascontiguousarray(feats, np.float32)).to(f'cuda:{device}')
    y = torch.empty(len(feats), dtype=torch.float32, device=x.device)
    model.forward(x.data_ptr(), len(feats), y.data_ptr())
    torch.cuda.synchronize()
    return y.cpu().numpy()


def evaluate(model: Optional[Mlp], recs: List[Dict]) -> Dict:
    """Regret t(choice) / t(best candidate) - 1 of the model's and of the root
    rule's choices."""
    rl, rh, wins = [], [], 0
    for r in recs:
        best = float(r['ms'].min())
        if model is not None:
            i = int(np.argmin(predict(model, r['feat'])))
            rl.append(float(r['ms'][i]) / best - 1.0)
        rh.append(r['heur_ms'] / best - 1.0)
        if model is not None and rl[-1] <= rh[-1] + 1e-12:
            wins += 1
    out = {'schemas': len(recs), 'heuristic_regret_mean': float(np.mean(rh)),
           'heuristic_regret_median': float(np.median(rh))}
    if model is not None:
        out.update(learned_regret_mean=float(np.mean(rl)), learned_regret_median=float(np.median(rl)),
                   learned_not_worse_frac=wins / max(1, len(recs)))
    return out


def save(model: Mlp, path: str, meta: Optional[Dict] = None):
    """Checkpoint: float32 parameters (.bin) + JSON meta with the normalisation."""
    model.get_params().tofile(path + '.bin')
    mean, std, ym, ys = model.norm
    with open(path + '.json', 'w') as f:
        json.dump({'in_dim': model.in_dim, 'hidden': model.hidden, 'mean': mean.tolist(), 'std': std.tolist(),
                   'y_mean': ym, 'y_std': ys, **(meta or {})}, f)


def load(path: str, device: int = 0) -> Mlp:
    with open(path + '.json') as f:
        m = json.load(f)
    model = Mlp(m['in_dim'], m['hidden'], 0, device)
    model.set_params(np.fromfile(path + '.bin', np.float32))
    model.set_norm(np.array(m['mean'], np.float32), np.array(m['std'], np.float32), m['y_mean'], m['y_std'])
    model.norm = (np.array(m['mean'], np.float32), np.array(m['std'], np.float32), m['y_mean'], m['y_std'])
    return model


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'costmodel_gb300')


def load_shipped(device: int = 0):
    """The checkpoint shipped with the package as (model, origin text), or
    (None, reason) when it is missing or was trained on another feature set;
    lmf_plan_learned with no model falls back to the root rule (Sec. 3.3)."""
    from .lmf import LMF_PLAN_FEATURES
    if not os.path.exists(SHIPPED + '.json') or not os.path.exists(SHIPPED + '.bin'):
        return None, 'rule (Sec. 3.3): no cost-model checkpoint'
    with open(SHIPPED + '.json') as f:
        meta = json.load(f)
    if meta.get('in_dim') != LMF_PLAN_FEATURES:
        return None, f"rule (Sec. 3.3): checkpoint has {meta.get('in_dim')} features, the planner {LMF_PLAN_FEATURES}"
    test = meta.get('test', {})
    return load(SHIPPED, device), (f"learned (cost-model checkpoint, {meta.get('train', {}).get('schemas')} "
                                   f"training schemas, held-out regret {test.get('learned_regret_mean')})")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument('--schemas', type=int, default=500)
    ap.add_argument('--train', type=int, default=400)
    ap.add_argument('--scale', type=float, default=0.1, help='fact-table size multiplier')
    ap.add_argument('--steps', type=int, default=3000)
    ap.add_argument('--threads', type=int, default=16, help='host threads compiling candidates')
    ap.add_argument('--out', default='')
    ap.add_argument('--records', default='', help='write every record (JSON) here')
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from workloads import config5_schema
    t0 = time.time()
    gen = (config5_schema(i, n_scale=args.scale) for i in range(args.schemas))
    recs = collect(gen, threads=args.threads, log=lambda s: print(s, file=sys.stderr, flush=True))
    if args.records:
        with open(args.records, 'w') as f:
            json.dump([{k: (v.tolist() if isinstance(v, np.ndarray) else v) for k, v in r.items()} for r in recs], f)
    t1 = time.time()
    tr, te = recs[:args.train], recs[args.train:]
    model, losses = train(tr, steps=args.steps)
    res = {'train': evaluate(model, tr), 'test': evaluate(model, te),
           'loss_first': float(np.mean(losses[:50])), 'loss_last': float(np.mean(losses[-50:])),
           'collect_s': t1 - t0, 'train_s': time.time() - t1, 'scale': args.scale,
           'candidates_mean': float(np.mean([len(r['ms']) for r in recs]))}
    print(json.dumps(res), flush=True)
    if args.out:
        save(model, args.out, meta=res)
    return 0


if __name__ == '__main__':
    sys.exit(main())
