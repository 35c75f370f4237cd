"""CPU reference of the dual-tree method as this library restates it for a
breadth-first, data-parallel traversal.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy and Python
loops; it shares no code with the CUDA path.  It serves two purposes:

 1. the tree partition and the per-iteration pair decisions it produces are
    the bit-exact reference for the GPU's kd-tree build and frontier;
 2. its own estimate G~ (every approximation evaluated in FP64 with the
    series reference, every leaf-leaf pair summed exactly) is checked against
    the exhaustive oracle, which pins its error control to Theorem 2.

The traversal follows the paper's DITO procedure (Fig. 7) and its pieces:
FD pruning (Section 5), bestMethod (Fig. 6) over DH / DL / H2L with the Lemma
4-6 bounds, the Theorem 2 rule with the W_T token scheme, exhaustive leaf-leaf
base cases (DITOBase) and recursion into child pairs, and the breadth-first
post-pass (Fig. 8).  Where the paper is silent this reference takes these
readings:

  * kd-tree: complete binary tree of depth d = min{k : ceil(n/2^k) <= L};
    node (k, i) holds sorted positions [floor(i n/2^k), floor((i+1) n/2^k));
    a node splits on its widest bounding-box dimension (lowest index on
    ties) and its left child takes the smallest points by the key
    (coordinate, original index); partitions are stable, so the points of
    every node stay in ascending original-index order;
  * node centre = bounding-box centre, r = half the widest extent;
  * iteration t holds pairs (Q, R, j) with Q at depth min(t, dQ) and R at
    depth min(t, dR); a pair that is neither pruned nor a leaf-leaf base case
    splits into its child pairs (both sides when both are internal);
  * the lower bound G^min of a group (Q, j) is the sum of W_R K(delta_max)
    over every pair that covers Q (finished at Q or an ancestor, or in the
    current frontier), raised to w_min(Q) in the monochromatic case and to
    the floor 2^floor_log2 W;
  * tokens: the group's token is split over its pairs in proportion to W_R;
    each pair spends or banks from its share (need = W E / (eps G) - W_R),
    leaf-leaf base cases bank W_R, splits return their share; children
    inherit a copy of their parent's token and finished lower bound;
  * all group sums use one fixed order: 32 strided partial sums followed by
    an xor butterfly over the 32 partials;
  * the per-pair kernel bounds are FP32 with rigorous relative margins (an
    exp2 written for this purpose, identically on both sides); everything
    that sums or compares budgets is FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import exhaustive as _ex
from . import mlp as _mlp
from . import series as _S

# --------------------------------------------------------------------------
# 2^x in FP32 for -125 <= x <= 0: x = k + f with k = rint(x), |f| <= 1/2,
# 2^f by Horner on its degree-7 Taylor polynomial in f (coefficients
# ln2^n / n!, truncation below 2^-27), times 2^k applied exactly.  Every
# operation is a single IEEE round-to-nearest FP32 operation.  Its relative
# error stays below 2^-20, which the bound margins below cover.
# --------------------------------------------------------------------------
def _exp2_coeffs():
    c, t = [], 1.0
    for n in range(8):
        c.append(np.float32(t))
        t = (t * 0.6931471805599453) / float(n + 1)
    return c


E2C = _exp2_coeffs()
F32_LO18 = np.float32(1.0 - 2.0 ** -18)
F32_HI18 = np.float32(1.0 + 2.0 ** -18)
F32_LO20 = np.float32(1.0 - 2.0 ** -20)
F32_HI20 = np.float32(1.0 + 2.0 ** -20)
F32_TINY = np.float32(2.0 ** -125)
F32_AMAX = np.float32(125.0)


def exp2_f32(x):
    x = np.asarray(x, np.float32)
    k = np.rint(x)
    f = x - k
    p = np.full(x.shape, E2C[7], dtype=np.float32)
    for n in range(6, -1, -1):
        p = p * f + E2C[n]
    return np.ldexp(p, k.astype(np.int32)).astype(np.float32)


def kernel_bounds(qt, rt, pq, pr, c32):
    """Rigorous FP32 bounds of the kernel over a node pair (Section 5's
    delta_min / delta_max from the bounding boxes): returns (K(delta_max)
    lower bound, K(delta_min) upper bound, e^{-delta_min^2 / 4h^2} upper
    bound).  The boxes are rounded outward to FP32; squared distances,
    exponent arguments and exponentials carry relative margins of 2^-18,
    2^-20 and 2^-18, each larger than the rounding they cover."""
    D = qt.D
    gsum = np.zeros(pq.size, np.float32)
    fsum = np.zeros(pq.size, np.float32)
    for d in range(D):
        ql, qh = qt.lo32[pq, d], qt.hi32[pq, d]
        rl, rh = rt.lo32[pr, d], rt.hi32[pr, d]
        g = np.maximum(np.float32(0), np.maximum(rl - qh, ql - rh))
        f = np.maximum(qh - rl, rh - ql)
        gsum = gsum + g * g
        fsum = fsum + f * f
    dmin2 = gsum * F32_LO18
    dmax2 = fsum * F32_HI18
    amax = (dmax2 * c32) * F32_HI20
    amin = (dmin2 * c32) * F32_LO20
    a4 = amin * np.float32(0.5)
    kmax = np.where(amax > F32_AMAX, np.float32(0), exp2_f32(-np.minimum(amax, F32_AMAX)) * F32_LO18)
    kmin = np.where(amin > F32_AMAX, F32_TINY, exp2_f32(-np.minimum(amin, F32_AMAX)) * F32_HI18)
    e4 = np.where(a4 > F32_AMAX, F32_TINY, exp2_f32(-np.minimum(a4, F32_AMAX)) * F32_HI18)
    return kmax.astype(np.float32), kmin.astype(np.float32), e4.astype(np.float32)


# --------------------------------------------------------------------------
# Fixed-order group reduction: 32 strided partials, then xor butterfly.
# --------------------------------------------------------------------------
def f32_mul_dir(a, b, up: bool):
    """a * b for FP32 arrays, rounded to FP32 toward -inf (up=False) or +inf.
    The FP64 product of two FP32 values is exact."""
    p = np.asarray(a, np.float32).astype(np.float64) * np.asarray(b, np.float32).astype(np.float64)
    return f32_up(p) if up else f32_down(p)


def f32_add_dir(a, b, up: bool):
    """a + b for FP32 arrays rounded to FP32 toward -inf / +inf: the exact
    sum is s + e with s the FP64 sum and e its error (Knuth's two-sum)."""
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    s = a + b
    bv = s - a
    e = (a - (s - bv)) + (b - bv)
    r = s.astype(np.float32)
    rd = r.astype(np.float64)
    if up:
        fix = (rd < s) | ((rd == s) & (e > 0))
        r[fix] = np.nextafter(r[fix], np.float32(np.inf))
    else:
        fix = (rd > s) | ((rd == s) & (e < 0))
        r[fix] = np.nextafter(r[fix], np.float32(-np.inf))
    return r


def group_reduce_f32(values, group_of, pos_in_group, ngroups: int, up: bool):
    """Per group: 32 lane-strided FP32 partial sums combined by the xor
    butterfly (the frontier kernel's order), every addition rounded in one
    direction; returned as FP64."""
    values = np.asarray(values, np.float32)
    acc = np.zeros((ngroups, 32), np.float32)
    lane = pos_in_group % 32
    rnd = pos_in_group // 32
    for k in range(int(rnd.max()) + 1 if rnd.size else 0):
        sel = rnd == k
        g, l = group_of[sel], lane[sel]
        acc[g, l] = f32_add_dir(acc[g, l], values[sel], up)
    for m in (16, 8, 4, 2, 1):
        acc = f32_add_dir(acc, acc[:, np.arange(32) ^ m], up)
    return acc[:, 0].astype(np.float64)


def group_reduce(values: np.ndarray, group_of: np.ndarray, pos_in_group: np.ndarray, ngroups: int):
    acc = np.zeros((ngroups, 32))
    lane = pos_in_group % 32
    order = np.lexsort((pos_in_group, group_of))       # sequential order within each lane
    np.add.at(acc, (group_of[order], lane[order]), values[order])
    for m in (16, 8, 4, 2, 1):
        acc = acc + acc[:, np.arange(32) ^ m]
    return acc[:, 0]


# --------------------------------------------------------------------------
# kd-tree
# --------------------------------------------------------------------------
def tree_depth(n: int, L: int) -> int:
    d = 0
    while -(-n // (1 << d)) > L:
        d += 1
    return d


def level_bounds(n: int, k: int) -> np.ndarray:
    nn = 1 << k
    return (np.arange(nn + 1, dtype=np.int64) * n) // nn


@dataclass
class Tree:
    n: int
    D: int
    depth: int
    perm: np.ndarray          # sorted position -> original index
    lo: np.ndarray            # (nodes, D) float64
    hi: np.ndarray
    lo32: np.ndarray          # lo rounded down to FP32
    hi32: np.ndarray          # hi rounded up to FP32
    center: np.ndarray
    rad: np.ndarray           # half the widest extent
    W: np.ndarray             # node weight sums
    wmin: np.ndarray
    begin: np.ndarray
    end: np.ndarray
    split_dim: np.ndarray     # -1 at leaves

    @property
    def nodes(self):
        return (1 << (self.depth + 1)) - 1
    W32d: np.ndarray = None   # W rounded down / up to FP32
    W32u: np.ndarray = None
    f32: bool = True          # the points are FP32 (not FP64)

    def __post_init__(self):
        self.W32d = f32_down(self.W)
        self.W32u = f32_up(self.W)


def build_tree(x: np.ndarray, w: np.ndarray, L: int) -> Tree:
    n, D = x.shape
    depth = tree_depth(n, L)
    perm = np.arange(n, dtype=np.int64)
    nodes = (1 << (depth + 1)) - 1
    split_dim = np.full(nodes, -1, dtype=np.int64)
    for k in range(depth):
        b = level_bounds(n, k)
        for i in range(1 << k):
            seg = perm[b[i]:b[i + 1]]
            pts = x[seg]
            ext = pts.max(0).astype(np.float64) - pts.min(0).astype(np.float64)
            s = int(np.argmax(ext))
            split_dim[(1 << k) - 1 + i] = s
            mid = ((2 * i + 1) * n) // (2 << k)
            order = np.lexsort((seg, pts[:, s]))        # by coordinate, then original index
            left = np.zeros(len(seg), dtype=bool)
            left[order[:mid - b[i]]] = True
            perm[b[i]:b[i + 1]] = np.concatenate([seg[left], seg[~left]])
    lo = np.zeros((nodes, D))
    hi = np.zeros((nodes, D))
    W = np.zeros(nodes)
    wmin = np.zeros(nodes)
    begin = np.zeros(nodes, dtype=np.int64)
    end = np.zeros(nodes, dtype=np.int64)
    for k in range(depth + 1):
        b = level_bounds(n, k)
        for i in range(1 << k):
            node = (1 << k) - 1 + i
            seg = perm[b[i]:b[i + 1]]
            begin[node], end[node] = b[i], b[i + 1]
            pts = x[seg]
            lo[node] = pts.min(0).astype(np.float64)
            hi[node] = pts.max(0).astype(np.float64)
            wmin[node] = float(np.min(w[seg]))
    # weights: sequential FP64 sums over each leaf, then pairwise up the tree
    b = level_bounds(n, depth)
    for i in range(1 << depth):
        node = (1 << depth) - 1 + i
        W[node] = float(np.cumsum(w[perm[b[i]:b[i + 1]]].astype(np.float64))[-1])
    for node in range((1 << depth) - 2, -1, -1):
        W[node] = W[2 * node + 1] + W[2 * node + 2]
    center = (lo + hi) * 0.5
    rad = ((hi - lo) * 0.5).max(axis=1)
    t = Tree(n, D, depth, perm, lo, hi, f32_down(lo), f32_up(hi), center, rad, W, wmin, begin, end,
             split_dim)
    t.f32 = x.dtype == np.float32
    return t


def f32_down(x):
    """Round FP64 values to FP32 toward -infinity."""
    f = np.asarray(x, np.float64).astype(np.float32)
    bad = f.astype(np.float64) > x
    f[bad] = np.nextafter(f[bad], np.float32(-np.inf))
    return f


def f32_up(x):
    """Round FP64 values to FP32 toward +infinity."""
    f = np.asarray(x, np.float64).astype(np.float32)
    bad = f.astype(np.float64) < x
    f[bad] = np.nextafter(f[bad], np.float32(np.inf))
    return f


# --------------------------------------------------------------------------
# error constants
# --------------------------------------------------------------------------
DEFAULT_PLIMIT = {1: 8, 2: 8, 3: 6, 4: 5, 5: 4, 6: 2}


def plimit_for(D: int) -> int:
    """Section 6 table (D=4 unstated: 5; D>6: 1; D=1 taken as 8)."""
    return DEFAULT_PLIMIT.get(D, 1)


TC_GUARD_LOG2 = -11     # absolute exponent error the tensor-core base case may add (log2 units)


def tc_enabled(D: int, f32: bool, nh: int, max_q_leaf: int, max_r_leaf: int, no_tc: bool = False) -> bool:
    """Whether the base case of a call may take its cross term from the
    tensor cores: 9 <= D <= 16, FP32 points, at most 32 bandwidths, leaves of
    at most 128 points."""
    return (not no_tc) and 9 <= D <= 16 and f32 and nh <= 32 and max_q_leaf <= 128 and max_r_leaf <= 128


def tc_rho() -> float:
    """Extra charge when the tensor-core base case is enabled: the expanded
    squared distance adds two roundings of the exponent argument (over
    exponents down to 2^-64: ln2 * 64 * 2u) and, on the leaf pairs its guard
    admits, an absolute exponent error of at most 2^TC_GUARD_LOG2 (ln2 times
    that)."""
    u = 2.0 ** -24
    return 0.6931471805599453 * (64.0 * 2.0 * u + 2.0 ** TC_GUARD_LOG2)


def fp32_rho(D: int, N: int, w_max: float, W: float, floor_log2: int, run: int, tc: bool = False) -> float:
    """A-priori relative error of the FP32 base case: per-term argument
    rounding for exponents down to 2^-64 (ln2 * 64 * (D+5) u: the squared
    distance (D+3) u relative -- the differences, the FMA chain, c -- the
    argument's FMA and the rounding of l = log2(w / w_max)), the ex2.approx
    bound 2^-21, FP32 recursive summation of positive terms over a run of at
    most `run` terms (one reference leaf: (run - 1) u) followed by the
    compensated sum across leaves (2 u), together (run + 1) u; terms below
    2^-64 w_max are charged absolutely against the floor."""
    u = 2.0 ** -24
    rho = 0.6931471805599453 * 64.0 * (D + 5) * u
    rho = rho + 2.0 ** -21
    rho = rho + float(run + 1) * u
    rho = rho + 2.0 ** (-63 - floor_log2) * ((N * w_max) / W)
    if tc:
        rho = rho + tc_rho()
    return rho


def bound_factor_table(D: int, P: int):
    F = [0.0] * (P + 1)
    BT = [0.0] * (P + 1)
    for p in range(1, P + 1):
        pp = p % D
        prod = math.factorial(p // D) ** (D - pp) * math.factorial(-(-p // D)) ** pp
        F[p] = float(math.comb(D + p - 1, D - 1)) / math.sqrt(float(prod))
        BT[p] = float(math.comb(D + p - 1, D))
    return F, BT


def rpow(r, p):
    out = np.ones_like(r)
    for _ in range(p):
        out = out * r
    return out


# --------------------------------------------------------------------------
# traversal
# --------------------------------------------------------------------------
FD, DH, DL, H2L, BASE, SPLIT = 0, 1, 2, 3, 4, 5
SEL_RULE, SEL_MLP, SEL_FD_ONLY, SEL_EXHAUSTIVE = 0, 1, 2, 3
SQRT2 = 1.4142135623730951
MLP_MIN_WORK = 2 ** 18      # the network is consulted for pairs with N_Q N_R at least this


@dataclass
class Traversal:
    iters: list = field(default_factory=list)   # per iteration: dict of arrays
    est: np.ndarray = None                       # (nodesQ, nh) FD estimates per node
    eps_t: float = 0.0
    rho: float = 0.0
    W: float = 0.0
    consulted: int = 0          # pairs scored by the selector network
    lookahead: int = 0          # pairs expanded ahead by the best-first ordering


COST_WEIGHTS = (32.0, 32.0, 32.0, 1.0)


def selector_features(qt, rt, q, r, j, kmin32, kmax32, share_t, kappa, inv_h, W, diam, t, P, D, cnt_q, cnt_r):
    """The 12 FP32 pair features of the selector network (same operations as
    the frontier kernel): plog2 of the kernel bounds, node sizes, the FD budget
    ratio (1 + share) / ((K(dmin) - K(dmax)) kappa / 2), radii / h, W_R / W,
    diameter / h; D, iteration and PLIMIT as numbers."""
    f32 = np.float32
    pl = _mlp.plog2_f32
    n = q.size
    X = np.empty((n, _mlp.NIN), f32)
    X[:, 0] = pl(kmin32)
    X[:, 1] = pl(kmax32)
    X[:, 2] = pl(cnt_q[q].astype(f32))
    X[:, 3] = pl(cnt_r[r].astype(f32))
    X[:, 4] = f32(D)
    hk = np.where(0.5 * kappa < 1e37, 0.5 * kappa, 1e37).astype(f32)
    thr = (1.0 + share_t).astype(f32)
    with np.errstate(divide="ignore", over="ignore"):
        X[:, 5] = pl((thr / ((kmin32 - kmax32).astype(f32) * hk).astype(f32)).astype(f32))
    X[:, 6] = pl((qt.rad[q] * inv_h[j]).astype(f32))
    X[:, 7] = pl((rt.rad[r] * inv_h[j]).astype(f32))
    X[:, 8] = pl((rt.W[r] / W).astype(f32))
    X[:, 9] = f32(t)
    X[:, 10] = pl((diam * inv_h[j]).astype(f32))
    X[:, 11] = f32(P)
    return X


def _argmax_certified(scores, certified):
    """Action 1..4 with the highest score among the certified ones (4 always
    is); ties go to the lowest action."""
    n = scores.shape[0]
    best = np.full(n, -1)
    bs = np.full(n, -np.inf, np.float32)
    for a in (1, 2, 3, 4):
        ok = np.ones(n, bool) if a == 4 else certified[a - 1]
        take = ok & ((best < 0) | (scores[:, a] > bs))
        best = np.where(take, a, best)
        bs = np.where(take, scores[:, a], bs)
    return best


def traverse(qt: Tree, rt: Tree, mono: bool, h, eps: float, plimit: int | None = None,
             selector: int = SEL_RULE, tokens: bool = True, floor_log2: int = -40,
             w_max: float = None, cost_weight=COST_WEIGHTS, mlp_params=None, no_tc: bool = False,
             best_first: bool = False):
    """Run the level-synchronous traversal; returns a Traversal whose iters[t]
    holds the frontier (q, r, j) and the decision (method, p, E) of every
    pair in the exact order the GPU processes them.

    bestMethod (Fig. 6) compares the paper's costs c_DH = N_Q D^{p+1},
    c_DL = N_R D^{p+1}, c_H2L = D^{2p+1} and c_Direct = D N_Q N_R, each
    multiplied by its weight in cost_weight (all ones: the paper's model).

    selector SEL_MLP: pairs whose FD test fails, that have a certified
    series method and whose N_Q N_R is at least MLP_MIN_WORK take the
    highest-scoring certified action of the selector network (mlp_params,
    oracle.mlp layout; ties: lowest action), split / base case counting as
    always certified; smaller such pairs keep the rule's choice.

    best_first: the best-first ordering of Section 1's priority-queue
    traversal, restricted to one level: in each (j, Q) group, the pairs whose
    bound gap W_R (K(delta_min) - K(delta_max)) is at least 1/8 of the group's
    total gap (the ones a queue ordered by gap pops first) are expanded on the
    reference side before the group is decided; the children's lower bound
    W_R1 K(delta_max(Q, R1)) + W_R2 K(delta_max(Q, R2)) replaces the pair's
    own in G^min (and in the finished lower bound) when it is larger."""
    kw = [float(v) for v in cost_weight]
    h = np.asarray(h, np.float64)
    nh = h.size
    D = qt.D
    P = plimit_for(D) if not plimit else plimit
    W = float(rt.W[0])
    floorW = W * 2.0 ** floor_log2
    run = -(-rt.n // (1 << rt.depth))          # largest reference leaf
    qrun = -(-qt.n // (1 << qt.depth))         # largest query leaf
    tc = tc_enabled(D, qt.f32, nh, qrun, run, no_tc)
    rho = fp32_rho(D, rt.n, w_max, W, floor_log2, run, tc)
    eps_t = eps - rho
    F, BT = bound_factor_table(D, P)
    Dpow = [1.0]
    for _ in range(2 * P + 1):
        Dpow.append(Dpow[-1] * float(D))
    c32 = (1.4426950408889634 / ((2.0 * h) * h)).astype(np.float32)   # log2(e) / 2h^2
    inv_h = 1.0 / h
    nQ = qt.nodes
    d2 = 0.0
    for d in range(D):
        d2 = d2 + (rt.hi[0, d] - rt.lo[0, d]) * (rt.hi[0, d] - rt.lo[0, d])
    diam = math.sqrt(d2)
    fin = np.zeros((nQ, nh))
    tok = np.zeros((nQ, nh))
    est = np.zeros((nQ, nh))
    cnt_q = (qt.end - qt.begin).astype(np.float64)
    cnt_r = (rt.end - rt.begin).astype(np.float64)

    pq = np.zeros(nh, dtype=np.int64)
    pr = np.zeros(nh, dtype=np.int64)
    pj = np.arange(nh, dtype=np.int64)
    out = Traversal(eps_t=eps_t, rho=rho, W=W)
    T = max(qt.depth, rt.depth)
    for t in range(T + 1):
        if pq.size == 0:
            break
        q_leaf = t >= qt.depth
        r_leaf = t >= rt.depth
        # groups: runs of equal (j, q) in the sorted frontier
        key_change = np.ones(pq.size, dtype=bool)
        key_change[1:] = (pq[1:] != pq[:-1]) | (pj[1:] != pj[:-1])
        gid = np.cumsum(key_change) - 1
        gstart = np.flatnonzero(key_change)
        ng = gstart.size
        pos = np.arange(pq.size) - gstart[gid]
        gq = pq[gstart]
        gj = pj[gstart]

        # per-pair kernel bounds (Section 5) in FP32 with rigorous margins
        kmax32, kmin32, e4_32 = kernel_bounds(qt, rt, pq, pr, c32[pj])
        kmax = kmax32.astype(np.float64)
        kmin = kmin32.astype(np.float64)
        WR = rt.W[pr]
        # the lower bound sum and the weight sum in FP32, rounded down and up
        dl32 = f32_mul_dir(rt.W32d[pr], kmax32, up=False)
        if best_first and not r_leaf:
            # gaps rounded to nearest in FP32, their group sum rounded up
            gap32 = rt.W32u[pr] * (kmin32 - kmax32)
            gtot = group_reduce_f32(gap32, gid, pos, ng, up=True).astype(np.float32)
            sel = np.flatnonzero((gap32 > 0) & (gap32 * np.float32(8.0) >= gtot[gid]))
            if sel.size:
                r1, r2 = 2 * pr[sel] + 1, 2 * pr[sel] + 2
                k1 = kernel_bounds(qt, rt, pq[sel], r1, c32[pj[sel]])[0]
                k2 = kernel_bounds(qt, rt, pq[sel], r2, c32[pj[sel]])[0]
                lc = f32_add_dir(f32_mul_dir(rt.W32d[r1], k1, up=False), f32_mul_dir(rt.W32d[r2], k2, up=False),
                                 up=False)
                dl32[sel] = np.maximum(dl32[sel], lc)
            out.lookahead += sel.size
        front = group_reduce_f32(dl32, gid, pos, ng, up=False)
        Wg = group_reduce_f32(rt.W32u[pr], gid, pos, ng, up=True)
        G = fin[gq, gj] + front
        if mono:
            G = np.maximum(G, qt.wmin[gq])
        G = np.maximum(G, floorW)
        Gp = G[gid]
        # per group: token per unit weight and the Theorem 2 scale W / (eps G)
        share = tok[gq, gj] / Wg
        kappa = W / (eps_t * G)
        allot = WR * share[gid] if tokens else np.zeros(pq.size)
        kap = kappa[gid]

        def need(E):
            return E * kap - WR

        e_fd = (WR * (kmin - kmax)) * 0.5
        est_fd = (WR * (kmin + kmax)) * 0.5
        method = np.full(pq.size, SPLIT if not (q_leaf and r_leaf) else BASE)
        porder = np.zeros(pq.size, dtype=np.int64)
        E = np.zeros(pq.size)
        n_fd = need(e_fd)
        use_fd = (n_fd <= allot) & (selector != SEL_EXHAUSTIVE)
        method[use_fd] = FD
        E[use_fd] = e_fd[use_fd]
        spent = np.where(use_fd, n_fd, 0.0)          # token needed by each pruned pair

        if selector in (SEL_RULE, SEL_MLP) and P >= 1:
            base = WR * e4_32.astype(np.float64)
            rR = rt.rad[pr] * inv_h[pj]
            rQ = qt.rad[pq] * inv_h[pj]
            best_c = np.full(pq.size, np.inf)
            best_m = np.full(pq.size, -1)
            best_p = np.zeros(pq.size, dtype=np.int64)
            best_need = np.zeros(pq.size)
            best_E = np.zeros(pq.size)
            x2 = SQRT2 * rQ
            cert = {}
            for m in (DH, DL, H2L):
                pm = np.zeros(pq.size, dtype=np.int64)
                needm = np.zeros(pq.size)
                Em = np.zeros(pq.size)
                for p in range(1, P + 1):
                    if m == DH:
                        Ep = (base * F[p]) * rpow(rR, p)
                    elif m == DL:
                        Ep = (base * F[p]) * rpow(rQ, p)
                    else:
                        expo = np.where(x2 <= 1.0, 0, p - 1)
                        tail = np.where(expo == 0, 1.0, rpow(x2, p - 1))
                        Ep = (base * F[p]) * (rpow(rQ, p) + (rpow(SQRT2 * rR, p) * BT[p]) * tail)
                    np_ = need(Ep)
                    ok = (pm == 0) & (np_ <= allot)
                    pm[ok] = p
                    needm[ok] = np_[ok]
                    Em[ok] = Ep[ok]
                found = pm > 0
                cert[m] = (pm, needm, Em)
                if m == DH:
                    c = (cnt_q[pq] * np.array([Dpow[p + 1] for p in pm])) * kw[0]
                elif m == DL:
                    c = (cnt_r[pr] * np.array([Dpow[p + 1] for p in pm])) * kw[1]
                else:
                    c = np.array([Dpow[2 * p + 1] for p in pm]) * kw[2]
                better = found & (c < best_c)
                best_c[better] = c[better]
                best_m[better] = m
                best_p[better] = pm[better]
                best_need[better] = needm[better]
                best_E[better] = Em[better]
            c_ex = ((float(D) * cnt_q[pq]) * cnt_r[pr]) * kw[3]
            if selector == SEL_RULE:
                series = (~use_fd) & (best_m >= 0) & (best_c <= c_ex)   # ties favour the series method (Fig. 6)
                method[series] = best_m[series]
                porder[series] = best_p[series]
                E[series] = best_E[series]
                spent = np.where(series, best_need, spent)
            else:
                contested = (~use_fd) & ((cert[DH][0] > 0) | (cert[DL][0] > 0) | (cert[H2L][0] > 0))
                consult = contested & (cnt_q[pq] * cnt_r[pr] >= MLP_MIN_WORK)
                # small pairs keep Fig. 6's choice
                series = contested & ~consult & (best_m >= 0) & (best_c <= c_ex)
                method[series] = best_m[series]
                porder[series] = best_p[series]
                E[series] = best_E[series]
                spent = np.where(series, best_need, spent)
                idx = np.flatnonzero(consult)
                out.consulted += idx.size
                if idx.size:
                    X = selector_features(qt, rt, pq[idx], pr[idx], pj[idx], kmin32[idx], kmax32[idx],
                                          (share if tokens else np.zeros(ng))[gid[idx]], kappa[gid[idx]], inv_h,
                                          W, diam, t, P, D, cnt_q, cnt_r)
                    sc = _mlp.infer_f32(mlp_params, X)
                    chosen = _argmax_certified(sc, [cert[a][0][idx] > 0 for a in (1, 2, 3)])
                    for a in (1, 2, 3):
                        sel = idx[chosen == a]
                        method[sel] = a
                        porder[sel] = cert[a][0][sel]
                        E[sel] = cert[a][2][sel]
                        spent[sel] = cert[a][1][sel]
        # Fig. 7's token update over the whole group: pruned pairs pay their
        # need (negative needs bank the excess), base cases bank W_R, splits
        # leave the token alone
        finished = method != SPLIT
        if tokens:
            banked = group_reduce_f32(np.where(method == BASE, rt.W32d[pr], np.float32(0)), gid, pos, ng, up=False)
            paid = group_reduce(spent, gid, pos, ng)
            tok_new = np.maximum(0.0, (tok[gq, gj] + banked) - paid)
        else:
            tok_new = np.zeros(ng)
        fin_add = front if (q_leaf and r_leaf) else \
            group_reduce_f32(np.where(finished, dl32, np.float32(0)), gid, pos, ng, up=False)
        est_add = group_reduce(np.where(method == FD, est_fd, 0.0), gid, pos, ng)
        fin[gq, gj] = fin[gq, gj] + fin_add
        tok[gq, gj] = tok_new
        est[gq, gj] = est[gq, gj] + est_add

        out.iters.append(dict(q=pq.copy(), r=pr.copy(), j=pj.copy(), method=method.copy(),
                              p=porder.copy(), E=E.copy(), G=Gp.copy()))

        # children of the split pairs, grouped by (j, child q) in sorted order
        sp = method == SPLIT
        if not sp.any():
            pq = pq[:0]
            break
        if not q_leaf:
            for g in range(ng):
                qn = gq[g]
                for c in (2 * qn + 1, 2 * qn + 2):
                    fin[c, gj[g]] = fin[qn, gj[g]]
                    tok[c, gj[g]] = tok[qn, gj[g]]
        nq_, nr_, nj_ = [], [], []
        gend = np.append(gstart[1:], pq.size)
        for g in range(ng):
            sel = np.flatnonzero(sp[gstart[g]:gend[g]]) + gstart[g]
            if sel.size == 0:
                continue
            rs = pr[sel]
            qn, jn = gq[g], gj[g]
            if not q_leaf and not r_leaf:
                for c in (2 * qn + 1, 2 * qn + 2):
                    rr = np.stack([2 * rs + 1, 2 * rs + 2], axis=1).ravel()
                    nq_.append(np.full(rr.size, c)); nr_.append(rr); nj_.append(np.full(rr.size, jn))
            elif q_leaf:
                rr = np.stack([2 * rs + 1, 2 * rs + 2], axis=1).ravel()
                nq_.append(np.full(rr.size, qn)); nr_.append(rr); nj_.append(np.full(rr.size, jn))
            else:
                for c in (2 * qn + 1, 2 * qn + 2):
                    nq_.append(np.full(rs.size, c)); nr_.append(rs.copy()); nj_.append(np.full(rs.size, jn))
        pq = np.concatenate(nq_)
        pr = np.concatenate(nr_)
        pj = np.concatenate(nj_)
    out.est = est
    return out


# --------------------------------------------------------------------------
# the estimate G~ in FP64 from a traversal (Fig. 7 actions + Fig. 8)
# --------------------------------------------------------------------------
def estimate(qt: Tree, rt: Tree, xq: np.ndarray, xr: np.ndarray, w: np.ndarray, h, trav: Traversal,
             plimit: int | None = None):
    """G~(x_q; h_j) in FP64, caller query order.  Also returns, per query
    and bandwidth, the sum of the error bounds charged to it."""
    h = np.asarray(h, np.float64)
    nh = h.size
    D = qt.D
    P = plimit_for(D) if not plimit else plimit
    M = xq.shape[0]
    Gs = np.zeros((qt.n, nh))                  # sorted query order
    charged = np.zeros((qt.n, nh))
    xqs = np.asarray(xq, np.float64)[qt.perm]
    T_P = _S.num_terms(D, P)
    B = np.zeros((qt.nodes, nh, T_P))

    def pts_r(node):
        idx = rt.perm[rt.begin[node]:rt.end[node]]
        return np.asarray(xr, np.float64)[idx], np.asarray(w, np.float64)[idx]

    for it in trav.iters:
        for q, r, j, m, p, E in zip(it["q"], it["r"], it["j"], it["method"], it["p"], it["E"]):
            b0, b1 = qt.begin[q], qt.end[q]
            if m in (FD, DH, DL, H2L):
                charged[b0:b1, j] += E
            if m == DH:
                xs, ws = pts_r(r)
                A = _S.hermite_coeffs(xs, ws, rt.center[r], h[j], p)
                Gs[b0:b1, j] += _S.eval_hermite(A, rt.center[r], h[j], xqs[b0:b1], p)
            elif m == DL:
                xs, ws = pts_r(r)
                Bl = _S.local_coeffs_direct(xs, ws, qt.center[q], h[j], p)
                B[q, j, :Bl.size] += Bl
            elif m == H2L:
                xs, ws = pts_r(r)
                A = _S.hermite_coeffs(xs, ws, rt.center[r], h[j], p)
                Bl = _S.h2l(A, rt.center[r], qt.center[q], h[j], p, p)
                B[q, j, :Bl.size] += Bl
            elif m == BASE:
                xs, ws = pts_r(r)
                Gs[b0:b1, j] += _ex.gauss_sum(xqs[b0:b1], xs, ws, [h[j]])[:, 0]
    # downward pass: FD estimates and local expansions to the leaves
    est = trav.est.copy()
    for node in range((1 << qt.depth) - 1):
        for c in (2 * node + 1, 2 * node + 2):
            est[c] += est[node]
            for j in range(nh):
                if np.any(B[node, j]):
                    B[c, j] += _S.l2l(B[node, j], qt.center[node], qt.center[c], h[j], P)
    leaf0 = (1 << qt.depth) - 1
    for i in range(1 << qt.depth):
        node = leaf0 + i
        b0, b1 = qt.begin[node], qt.end[node]
        for j in range(nh):
            Gs[b0:b1, j] += est[node, j]
            if np.any(B[node, j]):
                Gs[b0:b1, j] += _S.eval_local(B[node, j], qt.center[node], h[j], xqs[b0:b1], P)
    out = np.empty((M, nh))
    out[qt.perm] = Gs
    ch = np.empty((M, nh))
    ch[qt.perm] = charged
    return out, ch
