"""FP64 CPU oracle for TUCKET range-query Tucker decomposition (arXiv 2501.06647).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, literal NumPy
restatement of the paper's algorithms, used to check the CUDA engine.  Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import it; the engine (``paper_2501_06647_gb300``) never does,
and this package imports nothing from the engine.

Modules
-------
tensor   Appendix A: vec, mode-n matricization, mode-n product, Frobenius norm.
hooi     Section 2: Tucker-ALS (HOOI), Eq. (tuckerals) / Eq. (als-mat).
tree     Section 4.2 + Algorithms 3/4 (Insert/Append): the stream segment tree,
         and Algorithm 1 (Recall): the optimally pruned hit set (Section 5.1).
stitch   Eq. (partial-tucker) and Algorithm 2 (Stitch), Section 5.2, with the
         matricizations of Eq. (stitch-temp-2) and Eq. (stitch-nontemp-3).
metrics  Section 8.1: reconstruction error and the relative-error metric.
rng      the seeded random start of Algorithm 2 (splitmix64, Box-Muller, QR).
"""
from . import tensor, hooi, tree, stitch, metrics, rng  # noqa: F401
