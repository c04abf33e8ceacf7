"""CPU checks of the sparse list's bounce-back plan: the info word that the
host builds for every vector of the list (vector_info in clbm_host.h) and the
masked sparse step reads instead of working the plan out from the link bits
(halfway bounce-back, Sec. 4A).  A small host-only harness prints the words;
each field is checked here against the solid array itself: the pull source
of link i at node (x, y) is (x - e_ix, y - e_iy), periodic, and a node past
the row end counts as solid with every link bit set."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HARNESS = os.path.join(ROOT, "tests", "host", "vector_info_dump.cu")

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
OWN = [2, 4, 5, 6, 7, 8]        # links whose own-vector reads have slots, in slot order
LEFT = [1, 5, 8]                # neighbour elements a run's first node takes (e_x = +1)
RIGHT = [3, 6, 7]               # and its last node (e_x = -1)


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("vinfo")
    exe = str(d / "vector_info_dump")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-o", exe, HARNESS],
                   check=True, capture_output=True)

    def run(solid, V):
        ny, nx = solid.shape
        path = str(d / "solid.bin")
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(path)
        out = subprocess.run([exe, str(nx), str(ny), str(V), path], check=True, capture_output=True, text=True)
        words = np.array([int(w, 16) for w in out.stdout.split()], dtype=np.uint64)
        return words.reshape(ny, (nx + V - 1) // V)

    def rows(solid):
        ny, nx = solid.shape
        path = str(d / "solid.bin")
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(path)
        out = subprocess.run([exe, str(nx), str(ny), "0", path], check=True, capture_output=True, text=True)
        return out.stdout.split()
    def links(solid):
        ny, nx = solid.shape
        path = str(d / "solid.bin")
        np.ascontiguousarray(solid, dtype=np.uint8).tofile(path)
        out = subprocess.run([exe, str(nx), str(ny), "-1", path], check=True, capture_output=True, text=True)
        pairs = [[(int(t[:2], 16), int(t[2:], 16)) for t in line.split()] for line in out.stdout.splitlines()]
        return np.array(pairs, dtype=np.int64)          # [ny][nx][2]
    run.rows = rows
    run.links = links
    return run


def expected_fields(solid, y, v, V):
    """The plan of vector v of row y, from the solid array."""
    ny, nx = solid.shape

    def is_solid(xx, yy):
        return bool(solid[yy % ny, xx % nx])

    xs = [v * V + j for j in range(V)]
    inside = [x < nx for x in xs]
    node_solid = [not inside[j] or is_solid(xs[j], y) for j in range(V)]

    def link(j, i):            # the pull source of link i at node j is solid
        return not inside[j] or is_solid(xs[j] - EX[i], y - EY[i])
    rows = [all(not inside[j] or is_solid(xs[j], y + 1) for j in range(V)),      # e_y = -1: row y + 1
            all(node_solid),
            all(not inside[j] or is_solid(xs[j], y - 1) for j in range(V))]      # e_y = +1: row y - 1
    bounce = {i: any(link(j, i) and not node_solid[j] for j in range(V)) for i in range(1, 9)}
    cover = [bounce[i] and rows[EY[i] + 1] for i in OWN]
    rest = [bounce[i] and not rows[EY[i] + 1] for i in OWN]
    jr = min(V - 1, nx - 1 - v * V)
    left = [not node_solid[0] and not link(0, i) for i in LEFT]
    right = [not node_solid[jr] and not link(jr, i) for i in RIGHT]
    not_plain = any(node_solid) or any(link(j, i) for j in range(V) for i in range(1, 9))
    return dict(sflag=node_solid, rows=rows, cover=cover, rest=rest, b1=bounce[1], b3=bounce[3],
                left=left, right=right, not_plain=not_plain)


def fields_of(w, V):
    bits = lambda lo, n: [bool((w >> (lo + k)) & 1) for k in range(n)]
    return dict(sflag=bits(0, V), rows=bits(8, 3), cover=bits(11, 6), rest=bits(17, 6),
                b1=bool((w >> 23) & 1), b3=bool((w >> 24) & 1), left=bits(25, 3), right=bits(28, 3),
                not_plain=bool((w >> 31) & 1))


def lattices():
    rng = np.random.default_rng(1705)
    out = []
    for nx, ny, p in ((37, 11, 0.3), (64, 9, 0.15), (29, 6, 0.6), (8, 3, 0.5)):
        out.append((f"random {nx}x{ny} p={p}", (rng.random((ny, nx)) < p).astype(np.uint8)))
    sq = np.zeros((24, 48), dtype=np.uint8)
    x = np.arange(48) % 16
    yy = np.arange(24) % 12
    sq[(yy[:, None] < 6) & (x[None, :] < 8)] = 1
    out.append(("squares 48x24", sq))
    ch = np.zeros((9, 30), dtype=np.uint8)
    ch[0, :] = 1
    out.append(("channel 30x9", ch))
    return out


@pytest.mark.parametrize("V", [2, 4, 8])
def test_info_word_fields_match_the_solid_array(dump, V):
    for name, solid in lattices():
        words = dump(solid, V)
        ny, nvec = words.shape
        for y in range(ny):
            for v in range(nvec):
                got = fields_of(int(words[y, v]), V)
                exp = expected_fields(solid, y, v, V)
                assert got == exp, (name, V, y, v, hex(int(words[y, v])))


def test_bits_past_the_vector_width_are_clear(dump):
    """Solid-flag bits above V stay clear, so the step can take them as a mask."""
    for name, solid in lattices():
        words = dump(solid, 4)
        assert np.all((words & np.uint64(0xF0)) == 0), name


def test_cover_and_rest_split_the_bouncing_own_links(dump):
    """The own vectors held in plane slots and those in the lane's own slots
    never overlap; together they are the links 2, 4, 5, 6, 7, 8 that bounce
    at a fluid node of the vector."""
    for name, solid in lattices():
        words = dump(solid, 8)
        cover = (words >> np.uint64(11)) & np.uint64(0x3F)
        rest = (words >> np.uint64(17)) & np.uint64(0x3F)
        assert np.all((cover & rest) == 0), name


def test_open_lattice_vectors_are_plain(dump):
    """No solid node anywhere: every vector is plain (not-plain flag clear,
    no solid flags, no bounce-back reads) and fetches all six neighbour
    elements; the list itself stores 0 for such vectors, and the unmasked
    launch that steps them reads no info word."""
    words = dump(np.zeros((5, 40), dtype=np.uint8), 8)
    assert np.all(words == np.uint64(0x3F << 25))


def test_plain_row_range_is_the_longest_run_of_plain_rows(dump):
    """Rows of plain vectors (plain_rows: the sparse lattices' row list): a
    row is plain when no solid node lies in it or in the rows beside it
    (periodic); the batch's range (plain_row_range) is the longest run of
    them, empty when there is none."""
    rng = np.random.default_rng(17)
    cases = [("channel 30x9", np.pad(np.zeros((8, 30), np.uint8), ((1, 0), (0, 0)), constant_values=1)),
             ("open 16x5", np.zeros((5, 16), np.uint8)),
             ("all solid 7x4", np.ones((4, 7), np.uint8))]
    for k in range(12):
        ny, nx = int(rng.integers(3, 30)), int(rng.integers(1, 20))
        solid = np.zeros((ny, nx), np.uint8)
        for _ in range(int(rng.integers(0, 4))):
            solid[int(rng.integers(0, ny)), int(rng.integers(0, nx))] = 1
        cases.append((f"sparse rows {k}", solid))
    for name, solid in cases:
        ny = solid.shape[0]
        has = solid.any(axis=1)
        plain = [not (has[(y - 1) % ny] or has[y] or has[(y + 1) % ny]) for y in range(ny)]
        best = (0, 0)
        for a in range(ny):
            for b in range(a + 1, ny + 1):
                if all(plain[a:b]) and b - a > best[1] - best[0]:
                    best = (a, b)
        out = dump.rows(solid)
        got = tuple(int(v) for v in out[:2])
        assert got == best, (name, got, best)
        assert [c == "1" for c in out[2]] == plain, name


def test_link_bytes_of_the_masks_and_of_the_plan_agree(dump):
    """The kernels read the link bits that build_solid_masks uploads; the
    bounce-back plan is built from row_links.  Both give, for every node,
    bit i - 1 set where the pull source (x - e_ix, y - e_iy) is solid."""
    for name, solid in lattices():
        ny, nx = solid.shape
        got = dump.links(solid)
        expect = np.zeros((ny, nx), dtype=np.int64)
        for i in range(1, 9):
            src = np.roll(np.roll(solid, EY[i], axis=0), EX[i], axis=1)   # src[y, x] = solid[y - ey, x - ex]
            expect |= src.astype(np.int64) << (i - 1)
        assert np.array_equal(got[:, :, 0], expect), name
        assert np.array_equal(got[:, :, 1], expect), name
