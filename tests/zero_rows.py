"""Host count of the voxels in warp rows without off-diagonal entries (the
rows the one-term kernels evaluate as dt z + beta b), formed from D alone;
shared by the GPU tests."""
import numpy as np


def zero_row_voxels(D, op):
    """Voxels in warp rows (32 x-consecutive voxels) whose operator rows have no
    off-diagonal entry, from D alone: conservative faces vanish when either side
    has D = 0; literal faces towards +e carry D_p + D_q, towards -e 2 D_p."""
    nz, ny, nx = D.shape
    zero = np.ones(D.shape, dtype=bool)
    for ax in range(3):
        a = 2 - ax  # numpy axis of x, y, z
        n = D.shape[a]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[a] = slice(0, n - 1)
        hi[a] = slice(1, n)
        Dp, Dq = D[tuple(lo)], D[tuple(hi)]
        if op == "conservative":
            face = (Dp > 0) & (Dq > 0)  # the face between p and p + e
            zero[tuple(lo)] &= ~face
            zero[tuple(hi)] &= ~face
        else:
            zero[tuple(lo)] &= ~((Dp + Dq) > 0)  # towards +e
            zero[tuple(hi)] &= ~(Dq > 0)         # towards -e: 2 D_p of the voxel itself
    count = 0
    for x0 in range(0, nx, 32):
        seg = zero[:, :, x0:x0 + 32]
        rows = seg.all(axis=2)
        count += int(rows.sum()) * seg.shape[2]
    return count
