"""Host-side checks of the Newton-symmetric tiles' index arithmetic (no GPU).

The kernels map CTA t of a launch over nb blocks to the block pair (bi, bj),
bi <= bj, of the row-major upper triangle: row bi starts at bi*nb - bi(bi-1)/2;
the row comes from the closed-form root of that quadratic, corrected by one
step either way against rounding (sym_tile_of in sym_kernel.cuh). Every
particle of block b then receives exactly one partial per block ob. The TMA
copies of a block stay inside the blocked source buffer. These are the checks
made before the kernels first ran, kept as tests."""
import math
import random

import pytest


def tile_of(t, nb):
    a = 2.0 * nb + 1.0
    b = int((a - math.sqrt(a * a - 8.0 * t)) * 0.5)
    b = max(0, min(b, nb - 1))

    def start(r):
        return r * nb - r * (r - 1) // 2

    while b > 0 and start(b) > t:
        b -= 1
    while b + 1 < nb and start(b + 1) <= t:
        b += 1
    return b, b + (t - start(b))


@pytest.mark.parametrize("nb", list(range(1, 130)))
def test_every_block_pair_once(nb):
    seen = set()
    for t in range(nb * (nb + 1) // 2):
        bi, bj = tile_of(t, nb)
        assert 0 <= bi <= bj < nb
        seen.add((bi, bj))
    assert len(seen) == nb * (nb + 1) // 2


@pytest.mark.parametrize("nb", [256, 1024, 4096, 32768, 65535])
def test_large_block_counts_sampled(nb):
    rng = random.Random(nb)
    grid = nb * (nb + 1) // 2
    assert grid <= 2 ** 31 - 1
    for t in [0, 1, grid - 2, grid - 1] + [rng.randrange(grid) for _ in range(20000)]:
        bi, bj = tile_of(t, nb)
        assert 0 <= bi <= bj < nb
        assert bi * nb - bi * (bi - 1) // 2 + (bj - bi) == t


@pytest.mark.parametrize("n", [1, 2, 3, 511, 512, 513, 3001, 262144, 262145])
@pytest.mark.parametrize("B", [256, 512, 768, 1024])
def test_one_partial_per_block_and_copies_in_bounds(n, B):
    nb = (n + B - 1) // B
    P = B // 2
    writes = {}
    for t in range(nb * (nb + 1) // 2) if nb <= 64 else []:
        bi, bj = tile_of(t, nb)
        for p in range(bi * B, min(n, bi * B + B)):  # target side: slot bj
            writes.setdefault(p, []).append(bj)
        if bi != bj:
            for p in range(bj * B, min(n, bj * B + B)):  # source side: slot bi
                writes.setdefault(p, []).append(bi)
    for p, slots in writes.items():
        assert sorted(slots) == list(range(nb)), p
    # blocked source buffers (gravity 2, LJC 3, VJP 4, LJC VJP 5 arrays of P float4)
    for arrays in (2, 3, 4, 5):
        size = nb * arrays * P
        for bj in range(nb):
            npairs = (min(B, n - bj * B) + 1) // 2
            assert npairs <= P
            base = bj * arrays * P
            assert base + (arrays - 1) * P + npairs <= size


@pytest.mark.parametrize("n", [2, 3, 300, 511, 1025, 3001, 8192])
@pytest.mark.parametrize("B,S", [(512, 1), (512, 2), (512, 4), (1024, 8), (256, 4), (768, 2)])
def test_source_split_slots_match_the_finalize_rule(n, B, S):
    """With the source split, CTA (t, s) writes its targets' partial to slot
    bj*S + s and its part's sources' partial to slot bi*S + s; the finalize
    counts slot k of particle p iff k // S >= p // B or k % S is p's part. Every
    counted slot is written exactly once, no other slot is written, and the part
    copies stay inside the block."""
    nb = (n + B - 1) // B
    P = B // 2
    PS = P // S
    written = {}
    for t in range(nb * (nb + 1) // 2):
        bi, bj = tile_of(t, nb)
        nsrc = min(B, n - bj * B)
        for s in range(S):
            p0 = s * PS
            npairs = max(0, min(PS, (nsrc + 1) // 2 - p0))
            assert p0 + npairs <= P  # copy inside the block's arrays
            for p in range(bi * B, min(n, bi * B + B)):
                written.setdefault(p, []).append(bj * S + s)
            if bi != bj:
                nq = min(2 * npairs, nsrc - 2 * p0)
                for q in range(max(0, nq)):
                    written.setdefault(bj * B + 2 * p0 + q, []).append(bi * S + s)
    for p in range(n):
        own_b = p // B
        own_s = ((p - own_b * B) >> 1) // PS
        counted = [k for k in range(nb * S) if k // S >= own_b or k % S == own_s]
        assert sorted(written[p]) == counted, (p, sorted(written[p]), counted)
