"""Host-side checks of the kernels' work decompositions (no GPU): every face
record a sweep stores has exactly one owner thread, and every owner's index
stays inside its array.  The 3D x sweep stores (rather than adds) the
records it owns, with no zero fill before it, so a face it missed would keep
the previous step's value; the per-face x sweep's warp chunks likewise
write each x-face record once.  The ownership rules are restated from the
kernels (constants read from their headers) and enumerated for grid sizes
that put the chunk, block and segment edges in every position."""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1111_6583_gb300", "csrc")


def _const(header, name):
    with open(os.path.join(CSRC, header)) as f:
        m = re.search(r"constexpr int %s = (\d+);" % name, f.read())
    assert m, name
    return int(m.group(1))


XOWN = _const("classic3d.cuh", "kXOwn3d")
NW = _const("classic3d.cuh", "kXSweepLines")
ZSEG = _const("classic3d.cuh", "kZSeg3d")
CHUNK = _const("classic_faces.cuh", "kFacesChunk")


def xsweep3d_owners(nx, ny, nz):
    """(x-faces, y-face corrections, z-face corrections) stored by the 3D x
    sweep with transverse terms, as lists of (i, j, k) face indices."""
    nxc = (nx + XOWN - 1) // XOWN
    nyb = (ny + 1 + (NW - 2) - 1) // (NW - 2)
    nzs = (nz + 1 + ZSEG - 1) // ZSEG
    xf, yf, zf = [], [], []
    for bz in range(nzs):
        z0 = bz * ZSEG - 1
        z1 = min(z0 + ZSEG, nz)
        for by in range(nyb):
            for bx in range(nxc):
                x0 = bx * XOWN
                for w in range(NW):
                    j = by * (NW - 2) - 2 + w
                    owner_line = 1 <= w <= NW - 2 and j <= ny - 1
                    for lane in range(32):
                        f = x0 - 2 + lane
                        own_cell = 2 <= lane <= 29 and f <= nx - 1
                        own_face = (2 <= lane <= 29 and f <= nx) or (lane == 30 and f == nx)
                        for pz in range(z0 - 1, z1 + 1):
                            if owner_line and j >= 0 and own_face and 0 <= pz and z0 <= pz < z1:
                                xf.append((f, j, pz))
                            k = pz - 1
                            if owner_line and own_cell and k >= z0:
                                if k >= 0:
                                    yf.append((f, j + 1, k))
                                if j >= 0:
                                    zf.append((f, j, k + 1))
    return xf, yf, zf


@pytest.mark.parametrize("n3", [(56, 9, 31), (29, 10, 33), (5, 4, 4), (57, 21, 64), (28, 8, 32)])
def test_xsweep3d_writes_every_record_once(n3):
    nx, ny, nz = n3
    xf, yf, zf = xsweep3d_owners(nx, ny, nz)
    want_x = {(i, j, k) for i in range(nx + 1) for j in range(ny) for k in range(nz)}
    want_y = {(i, j, k) for i in range(nx) for j in range(ny + 1) for k in range(nz)}
    want_z = {(i, j, k) for i in range(nx) for j in range(ny) for k in range(nz + 1)}
    for got, want in ((xf, want_x), (yf, want_y), (zf, want_z)):
        assert len(got) == len(set(got)), "a record with two owners"
        assert set(got) == want


def faces_x_owners(nd, nx, ny):
    """Record indices the per-face x sweep's warp chunks store."""
    lines = ny + 2 if nd == 2 else 1
    cpl = (nx + 1 + CHUNK - 1) // CHUNK
    out = []
    for gw in range(cpl * lines):
        l = (gw // cpl) - 1 if nd == 2 else 0
        for lane in range(32):
            fraw = (gw % cpl) * CHUNK - 1 + lane
            f = min(fraw, nx + 1)
            # every load stays within the ghost layer
            assert -1 <= f <= nx + 1 and -2 <= f - 1
            if 1 <= lane <= CHUNK and fraw <= nx:
                out.append((l + (1 if nd == 2 else 0)) * (nx + 1) + fraw)
    return out


@pytest.mark.parametrize("nd,nx,ny", [(2, 59, 7), (2, 60, 3), (2, 61, 5), (1, 29, 1), (1, 90, 1),
                                      (2, 4, 4)])
def test_faces_x_chunks_write_every_record_once(nd, nx, ny):
    got = faces_x_owners(nd, nx, ny)
    nf = (nx + 1) * (ny + 2 if nd == 2 else 1)
    assert sorted(got) == list(range(nf))
