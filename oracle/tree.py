"""Stream segment tree (Section 4.2), Insert/Append (Algorithms 3 and 4) and
Recall (Algorithm 1).  TEST INFRASTRUCTURE ONLY: an explicit, pointer-based,
literal restatement in Python with FP64 NumPy payloads.

Node kinds (Section 4.2): leaf 'L', intermediate 'M', placeholder 'P'.  Node
ranges are kept in LEAF-BLOCK units; a leaf block is ``B`` consecutive slices
(B = 1 is the paper's tree exactly).

Readings of what the paper leaves open:
  * Leaf blocks.  The tree of Algorithms 3/4 is built over blocks of B slices;
    a leaf's payload is Tucker-ALS (``hooi.tucker_als``) of its raw block.
  * Open block.  When the first slice of block b arrives, Algorithm 4 (root
    extension) and the descent of Algorithm 3 run for block b, creating the
    leaf of block b as a "tail leaf"; its payload is Tucker-ALS of the raw
    slices received so far.  (It is computed lazily, when the block completes
    or before the next Recall: only its latest state can be observed, so this
    equals recomputing it after every append.)  When the block's last slice arrives, the
    descent of Algorithm 3 runs again and performs the deferred Stitch steps
    (a node v becomes intermediate when tau_v = b + 1).  With B = 1 both
    descents happen in the same append, which is Algorithm 3/4 verbatim.
  * Recall.  The theta test is done in integers, theta_den * overlap >=
    theta_num * |v| ("=" counts as a hit), with |v| in slices.  Leaves are
    terminal: a leaf that overlaps the query is a hit (with B = 1 every
    overlapping leaf passes the theta test anyway).  The tail leaf's range is
    [bB, T).
  * Stitch of a new intermediate node uses the build ranks, clamped by
    ``stitch.stitched_ranks``, and the tree's max_iter / tol.
"""
import numpy as np

from .hooi import tucker_als
from .stitch import partial_hit, stitched_ranks, stitch


class Node:
    __slots__ = ("sigma", "tau", "kind", "left", "right", "H", "V")

    def __init__(self, sigma, tau, kind):
        self.sigma = sigma        # range start, in blocks
        self.tau = tau            # range end (exclusive), in blocks
        self.kind = kind          # 'L', 'M' or 'P'
        self.left = None
        self.right = None
        self.H = None             # core tensor
        self.V = None             # [temporal factor, V^(2), ..., V^(p)]


class StreamSegmentTree:
    """Algorithms 3/4 over leaf blocks of ``B`` slices, payloads in FP64."""

    def __init__(self, dims, ranks, B=1, theta=(7, 10), max_iter=20, tol=0.01, init="hosvd", seed=0):
        self.dims = tuple(int(d) for d in dims)      # D_2..D_p
        self.ranks = tuple(int(r) for r in ranks)    # r_1..r_p (build ranks)
        self.p = len(self.ranks)
        assert self.p == len(self.dims) + 1 and self.p >= 2
        self.B = int(B)
        self.theta = (int(theta[0]), int(theta[1]))
        self.max_iter = int(max_iter)
        self.tol = float(tol)
        self.init = init           # Stitch start: "hosvd" or "random" (seeded, rng)
        self.seed = int(seed)
        self.T = 0                 # timespan in slices
        self.root = None
        self.tail = []             # raw slices of the open block
        self.tail_dirty = False    # tail leaf payload older than its raw slices
        self.stitch_count = 0      # number of Stitch calls made by appends

    # ----- helpers -------------------------------------------------------
    def slice_range(self, v):
        """[lo, hi) of node v in slices (the tail leaf ends at T)."""
        return v.sigma * self.B, min(v.tau * self.B, self.T)

    def _leaf_payload(self, block):
        G, U, _, _ = tucker_als(block, self.ranks, self.max_iter, self.tol)
        return G, U

    # ----- Algorithm 3 (Insert), in block units ---------------------------
    def _insert(self, v, b, complete):
        if v.sigma == b and v.tau == b + 1:
            v.kind = 'L'
            return v
        mu = (v.sigma + v.tau) // 2
        if b < mu:
            if v.left is None:
                v.left = Node(v.sigma, mu, 'P')
            return self._insert(v.left, b, complete)
        if v.right is None:
            v.right = Node(mu, v.tau, 'P')
        leaf = self._insert(v.right, b, complete)
        if complete and v.tau == b + 1:
            u1, u2 = v.left, v.right
            hits = [(u1.H, u1.V), (u2.H, u2.V)]
            r = stitched_ranks(hits, self.dims, self.ranks)
            G, U, _, _ = stitch(hits, r, self.max_iter, self.tol, self.init, self.seed)
            v.H, v.V = G, U
            v.kind = 'M'
            self.stitch_count += 1
        return leaf

    # ----- Algorithm 4 (Append), in block units ----------------------------
    def _append_block_start(self, b):
        if b == 0:
            self.root = Node(0, 1, 'P')
        elif b == self.root.tau:
            r2 = Node(0, 2 * self.root.tau, 'P')
            r2.left = self.root
            self.root = r2
        return self._insert(self.root, b, complete=False)

    def append(self, X_T):
        """Stream update (Section 3): append one slice X_T (shape D_2 x ... x D_p)."""
        X_T = np.asarray(X_T, dtype=np.float64)
        assert X_T.shape == self.dims
        b, off = divmod(self.T, self.B)
        if off == 0:
            self._append_block_start(b)
            self.tail = []
        self.tail.append(X_T)
        self.T += 1
        self.tail_dirty = True
        if off == self.B - 1:
            self._refresh_tail()
            self._insert(self.root, b, complete=True)
            self.tail = []

    def _refresh_tail(self):
        """Decompose the open (tail) leaf from its raw slices, if stale."""
        if self.tail_dirty and self.tail:
            leaf = self._find_leaf((self.T - 1) // self.B)
            leaf.H, leaf.V = self._leaf_payload(np.stack(self.tail, axis=0))
        self.tail_dirty = False

    def build(self, X):
        """T successive appends (the definition of building the tree over X)."""
        for t in range(np.asarray(X).shape[0]):
            self.append(X[t])

    def _find_leaf(self, b):
        v = self.root
        while not (v.sigma == b and v.tau == b + 1):
            mu = (v.sigma + v.tau) // 2
            v = v.left if b < mu else v.right
        return v

    # ----- Algorithm 1 (Recall) -------------------------------------------
    def recall(self, ts, te, v=None):
        """Pruned hit set of [ts, te) as a time-ordered list of nodes."""
        if v is None:
            self._refresh_tail()
            v = self.root
        lo, hi = self.slice_range(v)
        ov = max(0, min(te, hi) - max(ts, lo))
        tn, td = self.theta
        if v.kind == 'L' and ov > 0:
            return [v]
        if v.kind == 'M' and td * ov >= tn * (hi - lo):
            return [v]
        u1, u2 = v.left, v.right
        if te <= u1.tau * self.B:
            return self.recall(ts, te, u1)
        if ts >= u2.sigma * self.B:
            return self.recall(ts, te, u2)
        return self.recall(ts, te, u1) + self.recall(ts, te, u2)

    def hit_records(self, ts, te):
        """Hit set as integer records (level, index, node_lo, node_hi, clip_lo, clip_hi)."""
        out = []
        for v in self.recall(ts, te):
            lo, hi = self.slice_range(v)
            w = v.tau - v.sigma
            level = w.bit_length() - 1
            out.append((level, v.sigma >> level, lo, hi, max(ts, lo), min(te, hi)))
        return out

    # ----- Section 6.1: range query ---------------------------------------
    def hit_decompositions(self, ts, te):
        """(H~_i, V~_i) of every hit: stored payloads, or Eq. (partial-tucker) for partial hits."""
        hits = []
        for v in self.recall(ts, te):
            lo, hi = self.slice_range(v)
            a, b = max(ts, lo), min(te, hi)
            if a == lo and b == hi:
                hits.append((v.H, v.V))
            else:
                hits.append(partial_hit(v.H, v.V, a - lo, b - lo))
        return hits

    def query(self, ts, te, ranks=None, max_iter=None, tol=None):
        """Range query of Tucker decomposition over [ts, te) (Section 6.1).

        Returns dict(G, U, ranks, iters, errs, hits).
        """
        if not (0 <= ts < te <= self.T):
            raise ValueError("range outside [0, T)")
        req = self.ranks if ranks is None else tuple(int(r) for r in ranks)
        if any(a > b or a < 1 for a, b in zip(req, self.ranks)):
            raise ValueError("query ranks must be between 1 and the build ranks")
        hits = self.hit_decompositions(ts, te)
        r = stitched_ranks(hits, self.dims, req)
        G, U, it, errs = stitch(hits, r, self.max_iter if max_iter is None else max_iter,
                                self.tol if tol is None else tol, self.init, self.seed)
        return dict(G=G, U=U, ranks=r, iters=it, errs=errs, hits=self.hit_records(ts, te))

    # ----- introspection for invariants -----------------------------------
    def nodes(self):
        out, stack = [], ([self.root] if self.root is not None else [])
        while stack:
            v = stack.pop()
            out.append(v)
            for c in (v.left, v.right):
                if c is not None:
                    stack.append(c)
        return out

    def height(self):
        def h(v):
            if v is None:
                return 0
            return 1 + max(h(v.left), h(v.right))
        return h(self.root)
