"""Host-side model of the stage kernel's halo-ring copy (csrc/dg_kernels.cuh,
S0 halo) at the degrees where an element's modes are not a multiple of 16
bytes (0, 2, 4): ring element h gets a shared-memory slot of RS values that
starts on a 16-byte boundary, and the copy takes the 16-byte blocks from the
one holding the element's first value while they still hold some of its
values.  For every tile of a set of whole meshes, latitude bands (ghost rows
before row 0 and after the last row) and ensemble members (128-byte aligned
offsets in one array), every block read must lie inside the array padded to a
multiple of 16 bytes, every write inside the ring region, and every value of
every ring element must land at slot + (its address mod 16 bytes)."""
import pytest

CASES = [(4, 1), (4, 3), (4, 5), (8, 1), (8, 3), (8, 5)]   # (sizeof T, N = degree + 1)
MESHES = [(1, 3), (2, 9), (4, 2), (15, 19), (20, 10), (35, 19), (44, 14), (67, 19), (7, 5), (13, 11)]


def ring_slot(T, N):
    EL, VA = 3 * N * N, 16 // T
    rs = (EL + 2 * (VA - 1)) // VA * VA
    return rs if (rs // VA) % 2 else rs + VA      # an odd number of 16-byte blocks


def check_mesh(T, N, W, nlon, nlat, gs, gn, member_off=0):
    G, EL, VA = 32 // N, 3 * N * N, 16 // T
    RS = ring_slot(T, N)
    PPS = RS // VA
    cap = (2 * W + 2 * G) * RS
    row = nlon * EL
    total = (nlat + gs + gn) * row
    end = member_off + ((total * T + 15) // 16 * 16) // T   # padded array end, in values
    base = member_off + gs * row                             # own row 0
    pieces = 0
    for by in range((nlat + W - 1) // W):
        for bx in range((nlon + G - 1) // G):
            i0, j0 = bx * G, by * W
            Gv, Wv = min(G, nlon - i0), min(W, nlat - j0)
            nSe = Gv if (j0 > 0 or gs) else 0
            nNe = Gv if (j0 + Wv < nlat or gn) else 0
            nH = 2 * Wv + nSe + nNe
            iW = i0 - 1 if i0 > 0 else nlon - 1
            iE = i0 + Gv if i0 + Gv < nlon else 0

            def ring_off(h):
                if h < 2 * Wv:
                    east = h >= Wv
                    return ((j0 + (h - Wv if east else h)) * nlon + (iE if east else iW)) * EL
                r = h - 2 * Wv
                north = r >= nSe
                return ((j0 + Wv if north else j0 - 1) * nlon + i0 + (r - nSe if north else r)) * EL

            landed = {}
            for v in range(nH * PPS):
                h, c = divmod(v, PPS)
                src = base + ring_off(h)
                lead = src % VA
                if c * VA < lead + EL:
                    rd, dst = src - lead + c * VA, h * RS + c * VA
                    assert member_off <= rd and rd + VA <= end, (T, N, W, nlon, nlat, gs, gn, bx, by, h, c)
                    assert 0 <= dst and dst + VA <= cap
                    for q in range(VA):
                        landed[dst + q] = rd + q
                    pieces += 1
            for h in range(nH):
                src = base + ring_off(h)
                for q in range(EL):
                    assert landed[h * RS + src % VA + q] == src + q
    return pieces


@pytest.mark.parametrize("T,N", CASES)
def test_aligned_ring_copy_stays_inside_the_arrays(T, N):
    assert ring_slot(T, N) % (16 // T) == 0 and ring_slot(T, N) >= 3 * N * N + 16 // T - 1
    n = 0
    for W in (4, 8, 12):
        for nlon, nlat in MESHES:
            for gs, gn in [(0, 0), (1, 0), (0, 1), (1, 1)]:
                n += check_mesh(T, N, W, nlon, nlat, gs, gn)
        for off in (32, 96, 160):                     # ensemble members: 128-byte aligned offsets
            n += check_mesh(T, N, W, 13, 7, 0, 0, member_off=off)
    assert n > 0
