"""Host re-enactment of the coupling kernel's index arithmetic (no GPU).

compute-sanitizer is not available for these kernels, so the index arithmetic of
the tensor-core path's coupling kernel (`vterm_kernel`) is replayed here in numpy
for every launch shape the library reports (heom_tc_shape_params), on ragged
sizes and on several parameter sets concatenated in one launch:

  * block -> (set, branch, group of ADOs, band) as the kernel decodes it, with
    C's truncating division where the numerator can be negative;
  * every source load (union member m, rows a0 + groups j, column b) lies inside
    member m's d x d matrix of the block's branch;
  * every element of every output item is written exactly once;
  * every bulk L2 prefetch region lies inside one d x d matrix.

The union lists are built here from the hierarchy's own neighbour relation (each
ADO with its up- and down-neighbours), the definition the library's tables follow.

The tensor-core kernel's producer and epilogue thread mappings are replayed too:
every element of a d x d item (d <= 128) lands exactly once, at its 128-byte-swizzle
offset inside its 64 KB operand tile, and every element of tpart is stored once.
"""
import itertools

import numpy as np
import pytest

H = pytest.importorskip("paper_2601_20550_gb300.heom")


def hierarchy(D, L):
    """ADO index vectors with sum <= L and their neighbour sets (n +- e_j)."""
    ados = [a for a in itertools.product(range(L + 1), repeat=D) if sum(a) <= L]
    index = {a: i for i, a in enumerate(ados)}
    nbs = []
    for a in ados:
        s = set()
        for j in range(D):
            for step in (1, -1):
                b = list(a)
                b[j] += step
                b = tuple(b)
                if b in index:
                    s.add(index[b])
        nbs.append(s)
    return len(ados), nbs


def unions(n_ado, nbs, G):
    out = []
    for g in range((n_ado + G - 1) // G):
        s = set()
        for n in range(g * G, min(g * G + G, n_ado)):
            s.add(n)
            s |= nbs[n]
        out.append(sorted(s))
    return out


def cdiv(num, den):
    """C integer division (truncation toward zero) for a positive divisor."""
    return np.where(num >= 0, num // den, -((-num) // den))


def replay(sets, rpt, groups, G, pf):
    """sets: list of (d, n_ado, branches, nbs).  Returns per-set write counts."""
    rows = rpt * groups
    threads = 128 * groups
    meta, vt_begin = [], 0
    for d, n_ado, branches, nbs in sets:
        bands = (d + rows - 1) // rows
        gpb = (n_ado + G - 1) // G
        U = unions(n_ado, nbs, G)
        meta.append((d, n_ado, branches, bands, gpb, U, vt_begin))
        vt_begin += branches * gpb * bands
    total_blocks = vt_begin
    counts = [np.zeros(br * n * d * d, dtype=np.int64) for d, n, br, _ in sets]
    blk_all = np.arange(total_blocks)
    begins = np.array([m[6] for m in meta])
    ks_all = np.searchsorted(begins, blk_all, side="right") - 1
    for ks, (d, n_ado, branches, bands, gpb, U, vb) in enumerate(meta):
        blk = (blk_all[ks_all == ks] - vb)[:, None]
        if blk.size == 0:
            continue
        dd = d * d
        tid = np.arange(threads)[None, :]
        gi = blk // bands
        band = blk - gi * bands
        br = gi // gpb
        g = gi - br * gpb
        n0 = g * G
        assert (br < branches).all() and (g < gpb).all()
        b = tid & 127
        par = tid >> 7
        a0 = band * rows + par
        nrow = np.where(b < d, np.maximum(0, np.minimum(rpt, cdiv(d - a0 + groups - 1, groups))), 0)
        e0 = a0 * d + b
        es = groups * d
        maxu = max(len(u) for u in U)
        Upad = np.full((gpb, maxu), -1)
        for i, u in enumerate(U):
            Upad[i, :len(u)] = u
        # source loads of every union member, inside the member's matrix of this branch
        for s in range(maxu):
            m = Upad[g[:, 0], s][:, None]
            for j in range(rpt):
                act = (j < nrow) & (m >= 0)
                row = a0 + groups * j
                off = m * dd + e0 + j * es
                assert ((row < d) & (b < d))[act].all()
                assert ((off >= m * dd) & (off < (m + 1) * dd))[np.broadcast_to(act, off.shape)].all()
                assert (off[act] == (m * dd + row * d + b)[act]).all()
        # outputs: every element of every item written exactly once
        for k in range(G):
            n = n0 + k
            for j in range(rpt):
                act = (j < nrow) & (n < n_ado)
                off = (br * n_ado + n) * dd + e0 + j * es
                np.add.at(counts[ks], off[act], 1)
        # bulk L2 prefetch regions (band rows of each member, and of y and tpart of each item)
        if pf:
            r0 = band[:, 0] * rows
            nr = np.minimum(rows, d - r0)
            live = nr > 0
            assert (r0[live] * d + nr[live] * d <= dd).all()
    return counts


SIZES = [
    # (d, (D, L), branches): ragged bands, ragged ADO groups, a single ADO, d = 1
    (125, (3, 2), 2),
    (128, (2, 2), 1),
    (27, (4, 3), 3),
    (6, (2, 1), 2),
    (1, (1, 1), 2),
]


@pytest.mark.parametrize("shape", range(17))
def test_coupling_kernel_indexing(shape):
    assert H.heom_tc_shape_count() == 17
    rpt, groups, G, flags = H.heom_tc_shape_params(shape)
    for d, (D, L), branches in SIZES:
        n_ado, nbs = hierarchy(D, L)
        (cnt,) = replay([(d, n_ado, branches, nbs)], rpt, groups, G, flags & 1)
        assert (cnt == 1).all(), (shape, d, n_ado)
    # three parameter sets of different basis size and hierarchy concatenated in one launch
    sets = []
    for d, (D, L), branches in (SIZES[2], SIZES[0], SIZES[3]):
        n_ado, nbs = hierarchy(D, L)
        sets.append((d, n_ado, branches, nbs))
    for cnt in replay(sets, rpt, groups, G, flags & 1):
        assert (cnt == 1).all()


def sw128(r, c, colblock_stride):
    """Byte offset of FP16 element (r, c) in a tile of 64-column blocks, 128-byte rows,
    16-byte chunks XOR-swizzled by the row mod 8 (the UMMA 128B-swizzle layout)."""
    return (c >> 6) * colblock_stride + r * 128 + ((((c & 63) >> 3) ^ (r & 7)) << 4) + ((c & 63) * 2 & 15)


@pytest.mark.parametrize("d", [1, 6, 27, 64, 125, 128])
def test_tensor_core_producer_and_epilogue_mapping(d):
    """The tensor-core kernel's 384 producer threads (column pair 2 cp, rows r0 + 6 g,
    g < 24, offsets row_ofs[g mod 4] + 3072 (g div 4)) write every element of a d x d
    item exactly once at its swizzled offset (real half; the imaginary half adds 16384),
    inside one 64 KB tile; the 128 epilogue lanes (column b) with row blocks of 16 store
    every element of tpart exactly once."""
    kZZ = 65536
    written = np.zeros((d, d), dtype=np.int64)
    for tid in range(384):
        cp, r0 = tid & 63, tid >> 6
        c = 2 * cp
        cc = c & 63
        row_ofs = [(c >> 6) * (kZZ // 2) + (r0 + 6 * u) * 128 + ((((cc >> 3) ^ ((r0 + 6 * u) & 7))) << 4)
                   + ((cc * 2) & 15) for u in range(4)]
        for g in range(24):
            a = r0 + 6 * g
            if not (c < d and a < d):
                continue
            o = row_ofs[g & 3] + 3072 * (g >> 2)
            assert o == sw128(a, c, kZZ // 2) and o + 16384 + 4 <= kZZ and o % 4 == 0
            assert sw128(a, c + 1, kZZ // 2) == o + 2           # the half2 holds columns c, c + 1
            written[a, c] += 1
            if c + 1 < d:
                written[a, c + 1] += 1
    assert (written == 1).all()
    stored = np.zeros((d, d), dtype=np.int64)
    for b in range(128):
        for a0 in range(0, d, 16):
            for jj in range(16):
                if b < d and a0 + jj < d:
                    stored[a0 + jj, b] += 1
    assert (stored == 1).all()
