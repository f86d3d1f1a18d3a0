"""Seeded random start of Stitch (Algorithm 2's "randomly initialize U^(2..p)").

TEST INFRASTRUCTURE ONLY.  The paper draws the initial non-temporal factors
at random without saying how; to compare the engine with this oracle the
draw must be the same on both sides, so it is a counter-based generator that
each side writes from its published definition:

  * splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
    generators", OOPSLA 2014; the 64-bit finalizer constants of Vigna's
    public-domain reference): output k of the stream seeded with s is
    mix(s + (k + 1) * 0x9E3779B97F4A7C15 mod 2^64), where mix(z) is
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
    z *= 0x94D049BB133111EB; z ^= z >> 31 (all mod 2^64);
  * uniform k = ((output k >> 11) + 1) * 2^-53, in (0, 1];
  * Box-Muller (Box and Muller, Ann. Math. Statist. 29, 1958): Gaussian e
    uses the uniforms u1 = uniform(2 * (e // 2)), u2 = uniform(2 * (e // 2) + 1)
    and is sqrt(-2 ln u1) * cos(2 pi u2) for even e, * sin(2 pi u2) for odd e;
  * mode n = 2..p (index n >= 1 here) draws a D_n x r_n matrix, row-major,
    from Gaussians off_n, off_n + 1, ..., with off_n = sum over the earlier
    non-temporal modes m of D_m r_m; its initial factor is the Q of its
    reduced QR (LAPACK).  Only the column space matters to Algorithm 2.
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK = (1 << 64) - 1


def splitmix64(seed, k):
    """Output k (0-based) of the splitmix64 stream seeded with `seed`."""
    z = (int(seed) + (int(k) + 1) * GAMMA) & MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def uniform(seed, k):
    """Uniform k in (0, 1] (53 bits)."""
    return ((splitmix64(seed, k) >> 11) + 1) * 2.0 ** -53


def gaussian(seed, e):
    """Gaussian number e of the stream (Box-Muller on uniforms 2(e//2), 2(e//2)+1)."""
    j = int(e) // 2
    u1 = uniform(seed, 2 * j)
    u2 = uniform(seed, 2 * j + 1)
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * (np.cos(2.0 * np.pi * u2) if int(e) % 2 == 0 else np.sin(2.0 * np.pi * u2))


def gaussian_matrix(seed, offset, rows, cols):
    """rows x cols matrix of Gaussians offset, offset + 1, ... (row-major)."""
    G = np.empty((int(rows), int(cols)), dtype=np.float64)
    for d in range(int(rows)):
        for c in range(int(cols)):
            G[d, c] = gaussian(seed, offset + d * cols + c)
    return G


def seeded_factors(dims, ranks, seed):
    """Initial U^(2..p) of a seeded Stitch: [None, U_2, ..., U_p], U_n the Q
    of the reduced QR of the mode's Gaussian matrix (dims: D_2..D_p, ranks:
    the stitch's output ranks r_1..r_p)."""
    p = len(ranks)
    U = [None] * p
    off = 0
    for n in range(1, p):
        D, r = int(dims[n - 1]), int(ranks[n])
        Q, _ = np.linalg.qr(gaussian_matrix(seed, off, D, r), mode="reduced")
        U[n] = Q
        off += D * r
    return U
