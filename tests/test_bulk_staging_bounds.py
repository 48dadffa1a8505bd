"""CPU check of the address arithmetic of the mixed path's bulk-staged y / z tiles
(k_face_mixed_t_body with BULK in csrc/kernels_mixed.cu), restated here from the kernel: for every
block of several grid shapes, every cp.async.bulk copy reads a 16-byte-aligned, 144-byte range
inside the W32 allocation (2 NW ncell floats plus 64 of slack) starting at or below the tile's first
column, the shared-memory index the cell differences read stays inside its 36-float row, the rows
phase 1b reads were copied, and the mbarrier's transaction count stays below 2^20 bytes."""
import pytest

NW = 6            # primitives per cell (rho, u, v, w, p, T)
ROW = 36          # floats per staged row


def _check(n, ndim, visc, base=0x7F0000000000):
    h = [3 if a < ndim else 0 for a in range(3)]
    p = [n[a] + 2 * h[a] for a in range(3)]
    sy, sz = p[0], p[0] * p[1]
    nc = p[0] * p[1] * p[2]
    alloc = (2 * NW * nc + 64) * 4
    nvw = 6 if visc else 5
    na, nd = 2 * nvw, 15 + 5
    nr = nd + 1
    blocks = 0
    for D in range(1, ndim):
        other = 2 if D == 1 else 1
        s = sy if D == 1 else sz
        so = sy if other == 1 else sz
        for bx in range((n[0] + 31) // 32):
            for by in range((n[D] + 14) // 15):
                for bz in range(n[other]):
                    blocks += 1
                    d0, dend, o = h[D] + 15 * by, h[D] + n[D], h[other] + bz
                    nvalid = min(nr, p[D] - (d0 - 3))
                    assert 1 <= nvalid and na * nvalid * ROW * 4 < 1 << 20
                    col0 = h[0] + 32 * bx + o * so
                    for ar in range(na):
                        row = ar if ar < nvw else NW + ar - nvw
                        for k in range(nvalid):
                            a = base + 4 * (row * nc + col0 + (d0 - 3 + k) * s)
                            a16 = a & ~15
                            assert base <= a16 and a16 + 4 * ROW <= base + alloc
                            assert a - a16 + 4 * 32 <= 4 * ROW           # lanes 0..31 inside the row
                    for k in range(nd):
                        j = d0 - 3 + k
                        if any(h[0] + 32 * bx + lane < h[0] + n[0] for lane in range(32)) and j + 1 <= dend + 2:
                            assert k + 1 < nvalid
    return blocks


@pytest.mark.parametrize("n,ndim", [((128, 128, 128), 3), ((13, 11, 9), 3), ((33, 31, 17), 3),
                                    ((1, 40, 40), 3), ((24, 16, 1), 2), ((300, 200, 1), 2),
                                    ((45, 23, 1), 2), ((37, 29, 21), 3)])
def test_bulk_copies_stay_inside_their_buffers(n, ndim):
    for visc in (True, False):
        assert _check(n, ndim, visc) > 0
