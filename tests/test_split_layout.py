"""CPU checks of the split-precision slice layout and of the pipelined kernel's
fragment addressing, written out in Python from the layout's definition
(k-piece-major planes, 16-byte pieces; ldmatrix delivers to lane l, for each
8x8 matrix i, row l // 4 and 32-bit word l % 4 of the 16-byte row whose
address lane 8i + (l % 8) supplied). For every block shape up to 32 and every
k step: the fragments the lanes receive are exactly the mma.sync operand
fragments of the padded operands (rows beyond the problem may hold anything),
and no address leaves the operand's slot. The slice producer's index formulas
give every position of both layouts exactly once."""
import numpy as np
import pytest

RNG = np.random.default_rng(0)


def plane(M, rows, s, wpp):
    """k-piece-major plane of a rows x s operand (pieces of wpp cells)."""
    P = -(-s // wpp)
    out = np.zeros(rows * P * wpp)
    for kp in range(P):
        for r in range(rows):
            for w in range(wpp):
                k = kp * wpp + w
                out[(kp * rows + r) * wpp + w] = M[r, k] if k < s else 0.0
    return out


def ldsm(mem, addrs, nmat, wpp):
    """ldmatrix .x1/.x2/.x4 on b16 cells: cells per 16-byte row = wpp."""
    per = wpp // 4  # cells per 32-bit register: 2 BF16 or 1 TF32
    regs = np.zeros((32, nmat, per))
    for i in range(nmat):
        rows = [mem[addrs[8 * i + j]: addrs[8 * i + j] + wpp] for j in range(8)]
        for l in range(32):
            regs[l, i] = rows[l // 4][(l % 4) * per:(l % 4) * per + per]
    return regs


def lane_offsets(Mp, Np, wpp):
    l = np.arange(32)
    ra, pa = (l & 7) + ((l >> 3) & 1) * 8, l >> 4
    rb, pb = (l & 7) + (l >> 4) * 8, (l >> 3) & 1
    return wpp * (pa * Mp + ra), wpp * (pb * Np + rb), wpp * ra


def a_frag(regs, half, wpp, step):
    """The 16 x step A operand a warp's registers hold (mma.sync row layout)."""
    A = np.full((16, step), np.nan)
    for l in range(32):
        g, t = l // 4, l % 4
        if wpp == 8:  # BF16: m16n8k16 (or k8 in half steps)
            A[g, 2 * t:2 * t + 2], A[g + 8, 2 * t:2 * t + 2] = regs[l, 0], regs[l, 1]
            if half:
                A[:, 8:] = 0.0
            else:
                A[g, 2 * t + 8:2 * t + 10], A[g + 8, 2 * t + 8:2 * t + 10] = regs[l, 2], regs[l, 3]
        else:  # TF32: m16n8k8 (or one k piece in half steps)
            A[g, t], A[g + 8, t] = regs[l, 0][0], regs[l, 1][0]
            if half:
                A[:, 4:] = 0.0
            else:
                A[g, t + 4], A[g + 8, t + 4] = regs[l, 2][0], regs[l, 3][0]
    return A


def b_frag(regs, half, wpp, step):
    """The step x 16 B operand (two 8-column tiles) the registers hold."""
    B = np.full((step, 16), np.nan)
    for l in range(32):
        g, t = l // 4, l % 4
        if wpp == 8:
            if half:
                B[2 * t:2 * t + 2, g], B[2 * t:2 * t + 2, g + 8] = regs[l, 0], regs[l, 1]
                B[8:, :] = 0.0
            else:
                B[2 * t:2 * t + 2, g], B[2 * t + 8:2 * t + 10, g] = regs[l, 0], regs[l, 1]
                B[2 * t:2 * t + 2, g + 8], B[2 * t + 8:2 * t + 10, g + 8] = regs[l, 2], regs[l, 3]
        else:
            if half:
                B[t, g], B[t, g + 8] = regs[l, 0][0], regs[l, 1][0]
                B[4:, :] = 0.0
            else:
                B[t, g], B[t + 4, g] = regs[l, 0][0], regs[l, 1][0]
                B[t, g + 8], B[t + 4, g + 8] = regs[l, 2][0], regs[l, 3][0]
    return B


def check_shape(prec, Mp, Np, s, slot_rows):
    wpp = 8 if prec == "bf16" else 4
    nsl = 3 if prec == "bf16" else 2
    step = 16 if prec == "bf16" else 8
    L = RNG.standard_normal((Mp, s))
    R = RNG.standard_normal((Np, s))
    opb = nsl * slot_rows * 32  # cells: k up to 32
    lp, rp = plane(L, Mp, s, wpp), plane(R, Np, s, wpp)
    mem = np.full(2 * opb, 7.0)  # finite filler beyond the planes
    q = nsl - 1  # the last plane: the farthest reads
    sL, sR = q * len(lp), opb + q * len(rp)
    mem[sL:sL + len(lp)], mem[sR:sR + len(rp)] = lp, rp
    oa, ob, oa2 = lane_offsets(Mp, Np, wpp)
    for kk in range(0, s, step):
        half = (s - kk) <= step // 2
        koL, koR = wpp * ((kk // wpp) * Mp), wpp * ((kk // wpp) * Np)
        for mt in range(slot_rows // 16):
            if 16 * mt >= Mp:
                continue
            addrs = sL + oa + koL + 16 * wpp * mt
            n = 16 if half else 32
            assert (addrs[:n] + wpp <= opb).all()
            A = a_frag(ldsm(mem, addrs, 2 if half else 4, wpp), half, wpp, step)
            rows = min(16, Mp - 16 * mt)
            exp = np.zeros((16, step))
            kmax = min(step, s - kk)
            exp[:rows, :kmax] = L[16 * mt:16 * mt + rows, kk:kk + kmax]
            assert np.array_equal(A[:rows], exp[:rows])
        for p2 in range(slot_rows // 16):
            if 16 * p2 >= Np:
                continue
            addrs = sR + (oa2 if half else ob) + koR + 16 * wpp * p2
            n = 16 if half else 32
            assert (addrs[:n] + wpp <= 2 * opb).all()
            B = b_frag(ldsm(mem, addrs, 2 if half else 4, wpp), half, wpp, step)
            cols = min(16, Np - 16 * p2)
            exp = np.zeros((step, 16))
            kmax = min(step, s - kk)
            exp[:kmax, :cols] = R[16 * p2:16 * p2 + cols, kk:kk + kmax].T
            assert np.array_equal(B[:, :cols], exp[:, :cols])


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_small_instance_fragments(prec):
    for Mp in range(1, 17):
        for Np in (1, 5, 8, 9, 13, 16):
            for s in (1, 3, 4, 5, 8, 9, 12, 13, 16, 17, 23, 24, 31, 32):
                check_shape(prec, Mp, Np, s, 16)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_large_instance_fragments(prec):
    for Mp in (1, 5, 9, 16, 17, 23, 31, 32):
        for Np in (1, 8, 13, 17, 24, 32):
            for s in (1, 4, 5, 9, 13, 16, 17, 23, 32):
                check_shape(prec, Mp, Np, s, 32)


def test_producer_writes_each_position_once():
    """Each value is split once, over the block padded to whole pieces in both
    directions, and written to the left layout (rows along the columns) and to
    the right layout (columns along the rows)."""
    for P in (8, 4):
        for r in range(1, 33):
            for c in range(1, 33):
                rp, cp = -(-r // P) * P, -(-c // P) * P
                left = np.full(r * cp, -1)
                right = np.full(c * rp, -1)
                for e in range(rp * cp):
                    yc, xr = divmod(e, rp)
                    v = xr + yc * r if (xr < r and yc < c) else -2
                    li = ((yc // P) * r + xr) * P + (yc % P)
                    ri = ((xr // P) * c + yc) * P + (xr % P)
                    if xr < r:
                        assert left[li] == -1
                        left[li] = v
                    if yc < c:
                        assert right[ri] == -1
                        right[ri] = v
                assert (left != -1).all() and (right != -1).all()
                # left: piece (kp, row) holds row `row`, k = columns kp*P .. kp*P+P-1
                for kp in range(cp // P):
                    for row in range(r):
                        for w in range(P):
                            k = kp * P + w
                            want = row + k * r if k < c else -2
                            assert left[(kp * r + row) * P + w] == want
