"""Shared-memory bank model of the pass kernels' tile layouts (host only).

A warp's shared-memory access takes as many wavefronts as the largest number
of distinct 32-bit words it requests from one of the 32 banks; an 8-byte
(complex64) or 16-byte (complex128, double-float) element occupies 2 or 4
consecutive words.  This models the layouts of ``pass_common.cuh`` (a mapping
LO gives thread tid and register r the tile element
(tid & (2^LO - 1)) | ((tid >> LO) << (LO + RB)) | (r << LO); exchanges use the
padded index u + (u >> RB); high-pass cost bytes sit at u + 16 (u >> (4 + RB)))
and checks that every exchange and every padded cost-byte load of the
mappings the kernels use takes the minimum number of wavefronts."""
import pytest

GEOS = {"complex64 forward": (13, 5, 2), "complex128 forward / backward": (12, 4, 4),
        "complex64 backward": (12, 4, 2)}  # (T, RB, 32-bit words per element)
# exchanges of the round lists (low 8 -> 0 -> RB or 5, high 8 -> 4) and their reverses
PAIRS = [(8, 0), (0, 8), (0, 4), (4, 0), (0, 5), (5, 0), (8, 4), (4, 8)]


def tile_elem(T, RB, LO, tid, r):
    return (tid & ((1 << LO) - 1)) | ((tid >> LO) << (LO + RB)) | (r << LO)


def wavefronts(words):
    banks = {}
    for w in words:
        banks.setdefault(w % 32, set()).add(w)
    return max(len(s) for s in banks.values())


def extra_wavefronts(T, RB, wpe, LO, index):
    """Wavefronts above the minimum over all warps and registers of one tile."""
    threads = 1 << (T - RB)
    ideal = max(1, wpe) if wpe >= 1 else 1
    extra = 0
    for w in range(threads // 32):
        for r in range(1 << RB):
            words = []
            for lane in range(32):
                u = index(tile_elem(T, RB, LO, 32 * w + lane, r))
                if wpe >= 1:
                    words += [u * wpe + k for k in range(wpe)]
                else:  # one byte: its word
                    words.append(u // 4)
            extra += wavefronts(words) - ideal
    return extra


@pytest.mark.parametrize("geo", list(GEOS))
def test_exchanges_take_the_minimum_wavefronts(geo):
    T, RB, wpe = GEOS[geo]
    for a, b in PAIRS:
        if max(a, b) + RB > T:
            continue
        for LO in (a, b):
            assert extra_wavefronts(T, RB, wpe, LO, lambda u: u + (u >> RB)) == 0, (geo, a, b, LO)
    # the load mapping reads the dense buffer the tile copies fill
    assert extra_wavefronts(T, RB, wpe, T - RB, lambda u: u) == 0


@pytest.mark.parametrize("geo", ["complex64 forward", "complex128 forward / backward"])
def test_padded_cost_bytes_are_conflict_free(geo):
    """The forward high passes' padded cost bytes (the backward passes keep the
    dense layout: the padding's extra offset made their fused kernels spill)."""
    T, RB, _ = GEOS[geo]
    padded = lambda u: u + ((u >> (4 + RB)) << 4)
    for LO in (4, T - RB):  # the last mapping of a high pass, the load mapping
        assert extra_wavefronts(T, RB, 0, LO, padded) == 0, (geo, LO)
    # the dense layout costs one extra wavefront on every load in mapping 4
    assert extra_wavefronts(T, RB, 0, 4, lambda u: u) == (1 << (T - RB)) // 32 * (1 << RB)
