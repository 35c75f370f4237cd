"""Learned pair selector: training data, training and the stored network.

The selector (GS_SEL_MLP) scores the certified actions of a node pair and
the traversal takes the best-scoring one; the rule of Fig. 6 is what it
replaces, and every action it may take is certified by the same bounds, so
the eps guarantee does not depend on the network.

Training is done by the library's own kernels: gs_selector_samples runs an
FD-only traversal that logs every pair and labels each pair that has a
certified series method with the action of least modelled cost (its
subtree's cost when split), and gs_mlp_train fits the network with Adam.
This module only marshals those calls and stores the result.

The cost model's unit costs (seconds per frontier pair, per base-case term,
per FP64 operation slot of each series kernel, per series action) are
measured on the GPU by `calibrate` from a rule traversal of each training
problem: its phase and kernel times over the work its trace records.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import gs

# (u_pair, u_base, u_dh, u_dl, u_h2l, u_act): seconds per frontier pair, per
# base-case term, per FP64 operation slot of the DH / DL / H2L kernels and per
# series action (see gs_selector_samples); `calibrate` measures them
UNIT_COSTS = (1.0e-10, 1.9e-13, 2.0e-12, 2.0e-12, 2.0e-12, 1.0e-9)
U_ACT = 1.0e-9


def _tp(D, p):
    c = 1.0
    for i in range(1, D + 1):
        c = c * (p - 1 + i) / i
    return c


def _node_size(node, n):
    node = node.astype(np.int64)
    depth = np.floor(np.log2(node + 1.0)).astype(np.int64)
    depth = np.where((np.int64(1) << (depth + 1)) - 1 <= node, depth + 1, depth)   # guard rounding
    i = node - ((np.int64(1) << depth) - 1)
    return ((i + 1) * n >> depth) - (i * n >> depth)


def h2l_units(D, p):
    """FP64 lane slots of one H2L action of order p (the kernel's three paths)."""
    T = _tp(D, p)
    if p == 1:
        return 4.0 * D + 30.0
    if p == 2:
        return 16.0 * D + 30.0
    if D == 3 and p <= 6:                      # the separable three-dimensional kernel
        return 2.0 * p * T + (0.5 * p * (p + 1)) ** 2 + 80.0
    if T <= 20 and D * (2 * p - 1) <= 32:
        return T * T * (D + 1.0) + T * D + 3.0 * D * (2 * p - 1) + 30.0
    return 32.0 * (np.ceil(T / 32.0) * T * (D + 1.0) + 40.0)


def dhdl_units(D, p, m):
    """FP64 lane slots per point of a DH (m = 1) or DL (m = 2) action of order p."""
    T = _tp(D, p)
    if m == 2 and T > 32:
        T = 32.0 * np.ceil(T / 32.0)
    return T * (D + 1.0) + 3.0 * D * p + 30.0


def calibrate(points, weights, h, eps, queries=None, opts=None):
    """Unit costs measured on this GPU from one rule traversal of the problem:
    phase and kernel times (gs_stats) over the work the traversal did (its
    trace: every series action with its order and node sizes)."""
    import torch
    q = points if queries is None else queries
    o = gs.gs_opts_default() if opts is None else opts
    st = gs.gs_stats()
    gs.gs_sum(q, points, weights, h, eps, opts=o)                      # warm
    torch.cuda.synchronize()
    gs.gs_sum(q, points, weights, h, eps, opts=o, stats=st)
    npairs = st.pairs_fd + st.pairs_dh + st.pairs_dl + st.pairs_h2l + st.pairs_base + st.pairs_split
    _, tr, _, _ = gs.gs_sum_trace(q, points, weights, h, eps, opts=o, trace_cap=int(npairs) + 16)
    t = tr.cpu().numpy().astype(np.int64)
    method = t[:, 3] & 0xff
    p = (t[:, 3] >> 8) & 0xff
    D = points.shape[1]
    M, N = q.shape[0], points.shape[0]
    u = list(UNIT_COSTS)
    u[0] = st.ms_phase[gs.GS_PH_FRONTIER] * 1e-3 / max(npairs, 1)
    u[1] = st.ms_phase[gs.GS_PH_BASE] * 1e-3 / max(st.point_pairs_base, 1)
    for k, m in enumerate((1, 2, 3)):
        sel = method == m
        cnt = int(sel.sum())
        if cnt == 0:
            continue
        pp = p[sel]
        if m == 3:
            units = float(sum(h2l_units(D, int(v)) for v in pp))
        else:
            nodes = _node_size(t[sel, 0], M) if m == 1 else _node_size(t[sel, 1], N)
            per = np.array([dhdl_units(D, int(v), m) for v in pp])
            units = float(np.sum(nodes * per))
        sec = st.ms_series[k] * 1e-3 - U_ACT * cnt
        if units > 0 and sec > 0:
            u[2 + k] = sec / units
    u[5] = U_ACT
    return tuple(u), st.as_dict()
PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_params.npy")
META_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_params.json")


def samples(points, weights, h, eps, queries=None, opts=None, units=UNIT_COSTS, cap=1 << 24):
    """Training samples of one problem (torch CUDA tensors x, y, s) and the
    modelled costs (cheapest policy, FD-only policy)."""
    q = points if queries is None else queries
    return gs.gs_selector_samples(q, points, weights, h, eps, units, cap, opts=opts)


def init_params(seed=0):
    """Random initial network (He initialisation), float32 numpy array."""
    g = np.random.default_rng(seed)
    nin, nh, nout = gs.GS_MLP_NIN, 64, gs.GS_MLP_NOUT
    parts = [np.zeros(nin), np.ones(nin), g.normal(0, np.sqrt(2.0 / nin), nin * nh), np.zeros(nh),
             g.normal(0, np.sqrt(2.0 / nh), nh * nh), np.zeros(nh), g.normal(0, np.sqrt(1.0 / nh), nh * nout),
             np.zeros(nout)]
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == gs.GS_MLP_NPARAM
    return p


def train(x, y, s=None, epochs=30, batch=4096, lr=2e-3, seed=0, init=None):
    """Fit a network to samples on the GPU; returns (params CUDA tensor, epoch losses)."""
    import torch
    p0 = init_params(seed) if init is None else np.asarray(init, np.float32)
    params = torch.from_numpy(p0).to(x.device)
    losses = gs.gs_mlp_train(params, x, y, s, epochs=epochs, batch=batch, lr=lr, seed=seed, set_norm=True)
    return params, losses


def options(params, base=None):
    """gs_opts selecting the learned ordering with the given device parameters."""
    o = gs.gs_opts_default() if base is None else base
    o.selector = gs.GS_SEL_MLP
    o.selector_params = params.data_ptr()
    return o


def save(params, meta=None, path=PARAMS_FILE):
    np.save(path, params.detach().cpu().numpy().astype(np.float32))
    if meta is not None:
        with open(os.path.splitext(path)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1, sort_keys=True)


def load(device="cuda", path=PARAMS_FILE):
    """The stored network as a CUDA tensor (raises if it was never trained)."""
    import torch
    if not os.path.exists(path):
        raise FileNotFoundError("no trained selector at %s; run python -m paper_1206_6857_gb300.selector" % path)
    return torch.from_numpy(np.load(path).astype(np.float32)).to(device)


def _training_problems():
    """Seeded training problems shaped like the workloads (a plain KDE sum in
    D = 2, a bandwidth sweep in D = 3, the series regime in D = 5, and
    uneven problems in D = 2..8), small enough to log every pair."""
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from workloads import synth
    yield synth.config1()
    yield synth.config2(scale=0.03)
    yield synth.config2(scale=0.1)
    yield synth.config2(scale=0.1, nh=8)
    yield synth.config3(scale=0.04, eps=1e-3)
    yield synth.config3(scale=0.1, eps=1e-2)
    for i in range(0, 40, 8):
        yield synth.config5_problem(i)


def _collect(problems, factors=(1.0, 1.0, 1.0)):
    """Samples of every problem; series unit costs from a rule run of the
    problem, multiplied by per-method factors (DH, DL, H2L)."""
    import torch
    xs, ys, ss, info = [], [], [], []
    for wl in problems:
        p = torch.from_numpy(np.ascontiguousarray(wl.refs)).cuda()
        w = torch.from_numpy(np.ascontiguousarray(wl.weights)).cuda()
        q = None if wl.mono else torch.from_numpy(np.ascontiguousarray(wl.queries)).cuda()
        o = gs.gs_opts_default()
        o.leaf_size = wl.leaf_size
        units, _ = calibrate(p, w, wl.h, wl.eps, queries=q, opts=o)
        units = tuple(units[:2]) + tuple(u * f for u, f in zip(units[2:5], factors)) + (units[5],)
        x, y, s, mc = samples(p, w, wl.h, wl.eps, queries=q, opts=o, units=units)
        xs.append(x)
        ys.append(y)
        ss.append(s)
        counts = np.bincount(y.cpu().numpy(), minlength=5).tolist()
        info.append({"workload": wl.name, "samples": int(x.shape[0]), "labels": counts, "unit_costs": units,
                     "model_cost_best": mc[0], "model_cost_fd_only": mc[1]})
        print(info[-1], flush=True)
    return torch.cat(xs), torch.cat(ys), torch.cat(ss), info


def main(epochs=40, rounds=4, out=PARAMS_FILE):
    """Collect samples from the training problems, train, store the network.

    The first pass takes the series unit costs measured on the rule's own actions.
    The learned policy then picks other actions (larger nodes, higher orders),
    so each further pass measures the unit costs again on a run of the
    current network over a calibration problem, scales every problem's series
    costs by the ratio to the rule's, relabels and retrains."""
    import sys
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from workloads import synth
    factors = (1.0, 1.0, 1.0)
    history = []
    params = None
    for rnd in range(rounds):
        x, y, s, info = _collect(_training_problems(), factors)
        params, losses = train(x, y, s, epochs=epochs)
        scores = gs.gs_mlp_forward(params, x)
        acc = float((scores[:, 1:].argmax(dim=1) + 1 == y).float().mean())
        history.append({"round": rnd, "factors": factors, "samples": int(x.shape[0]), "loss": losses[-1],
                        "train_accuracy": acc})
        print("round %d: %d samples, loss %.4f, accuracy %.3f, factors %s" % (rnd, x.shape[0], losses[-1], acc,
                                                                            factors), flush=True)
        if rnd + 1 < rounds:
            wl = synth.config2(scale=0.1)
            p = torch.from_numpy(np.ascontiguousarray(wl.refs)).cuda()
            w = torch.from_numpy(np.ascontiguousarray(wl.weights)).cuda()
            o = gs.gs_opts_default()
            o.leaf_size = wl.leaf_size
            u_rule, _ = calibrate(p, w, wl.h, wl.eps, opts=o)
            u_mlp, _ = calibrate(p, w, wl.h, wl.eps, opts=options(params, o))
            factors = tuple(max(1.0, f * um / ur) for f, um, ur in zip(factors, u_mlp[2:5], u_rule[2:5]))
    meta = {"problems": info, "epochs": epochs, "rounds": history, "loss": losses, "train_accuracy": acc}
    save(params, meta, out)
    print("trained on %d samples, final loss %.4f, accuracy %.3f" % (x.shape[0], losses[-1], acc))
    return params, meta


if __name__ == "__main__":
    from . import build
    build.build()
    main()
