"""Counter-based sampling spec of the oracle -- TEST INFRASTRUCTURE ONLY.

The paper draws blocks "randomly" (Algorithm 1, the selection step; Sec. 4
models it with random 0/1 diagonal matrices) without fixing a distribution.
Reading used on both sides of the parity tests: uniform without replacement
within an iteration, independent across iterations; weighted draws by inverse
CDF over FP64 weights.

Random numbers come from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014),
written here from its published definition: the n-th output (n >= 1) of the
generator seeded with s is mix(s + n * 0x9E3779B97F4A7C15 mod 2^64), where mix
is the variant-13 finaliser. Draw number (it * 2^20 + lane + 1) is the draw of
`lane` at iteration `it`; u = (out >> 11) * 2^-53 is uniform on [0, 1).
"""
MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
LANE_BITS = 20

# lanes used by the block sampler
LANE_ROWS = 0          # + t, t < alpha*M
LANE_COLS = 256        # + t, t < gamma*N
LANE_PAIR = 1024       # residual-weighted pair draw
LANE_CELLS = 2048      # + pair * n_views_in_block + view position


def mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix64(seed: int, n: int) -> int:
    """n-th output (n >= 1) of SplitMix64 seeded with `seed`."""
    return mix64((seed + n * GOLDEN) & MASK)


def uniform(seed: int, it: int, lane: int) -> float:
    n = (it << LANE_BITS) + lane + 1
    return (splitmix64(seed, n) >> 11) * (1.0 / 9007199254740992.0)


def choose_k_of_n(seed: int, it: int, lane0: int, n: int, k: int):
    """k distinct items of range(n): partial Fisher-Yates, the t-th swap
    partner is t + floor(u_t * (n - t)). Returned sorted ascending."""
    perm = list(range(n))
    for t in range(k):
        u = uniform(seed, it, lane0 + t)
        idx = t + int(u * (n - t))
        perm[t], perm[idx] = perm[idx], perm[t]
    return sorted(perm[:k])


def choose_weighted(u: float, w) -> int:
    """Smallest index whose running FP64 sum of weights exceeds u * total
    (weights summed in index order)."""
    total = 0.0
    for wi in w:
        total += float(wi)
    c = u * total
    acc = 0.0
    last = 0
    for i, wi in enumerate(w):
        acc += float(wi)
        if float(wi) > 0.0:
            last = i
        if acc > c:
            return i
    return last
