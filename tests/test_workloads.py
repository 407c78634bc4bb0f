"""Input recipes: element counts of every workload, outward orientation by
the divergence theorem (the signed volume a closed mesh encloses), door and
baffle labelling, and the placement of sources and receivers."""
import numpy as np

from paper_2103_16073_gb300 import workloads as W


def enclosed_volume(v, t):
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


def test_counts():
    assert W.cfg_small().n == 3072
    assert W.cfg_1khz().n == 39368
    assert W.cfg_1khz_sub().n == 3984
    assert W.cfg_baffle_sub().n == 3280
    assert W.cfg_largest(nrec=4).n == 2644104
    ir = W.ir_sweep(f_max=640.0, df=10.0)
    assert len(ir) == 64 and ir[0].n == 1440 and ir[-1].n == 81000
    assert all(a.n <= b.n for a, b in zip(ir, ir[1:]))


def test_orientation_and_volumes():
    v, t, _ = W.shoebox_mesh(3.0, 2.4, 2.0, 7, 6, 5)
    assert abs(enclosed_volume(v, t) - 3.0 * 2.4 * 2.0) < 1e-9
    v, t, _ = W.lroom_mesh(0.5)
    assert abs(enclosed_volume(v, t) - (5 * 4 * 3 + 3 * 3 * 3)) < 1e-9
    v, t, wall = W.baffle_room_mesh(0.35, 0.02)
    assert abs(enclosed_volume(v, t) - (60.0 - 0.02 * 2.0 * 1.5)) < 1e-9   # the box is outside the air
    v, t, wall = W.baffle_room_mesh(0.35, 0.0)
    assert abs(enclosed_volume(v[:], t[wall != W.WALL_BAFFLE]) - 60.0) < 1e-9
    sheet = t[wall == W.WALL_BAFFLE]
    nrm = np.cross(v[sheet[:, 1]] - v[sheet[:, 0]], v[sheet[:, 2]] - v[sheet[:, 0]])
    assert np.all(nrm[:, 0] > 0) and np.allclose(v[sheet][..., 0], W.BAFFLE_X)


def test_door_and_baffle_labels():
    wl = W.cfg_baffle_sub()
    v, t = wl.verts, wl.tris
    cen = v[t].mean(axis=1)
    door = wl.wall == W.WALL_DOOR
    assert door.any()
    assert np.all(np.abs(cen[door, 1]) < 1e-12)
    assert np.all((cen[door, 0] > W.DOOR_X[0]) & (cen[door, 0] < W.DOOR_X[1]) & (cen[door, 2] < W.DOOR_Z[1]))
    assert np.all(wl.beta[door] == 1.0) and np.all(wl.beta[wl.wall == W.WALL_BAFFLE] == 1.0)
    assert np.all(wl.beta[wl.wall < W.WALL_DOOR] == 0.2)


def test_sources_and_receivers_placement():
    wl = W.cfg_baffle(nsrc=8, nrec=64)
    pts = np.concatenate([wl.sources, wl.receivers])
    assert np.all(W.baffle_room_inside(pts, 0.25))
    d = np.linalg.norm(wl.receivers[:, None, :] - wl.sources[None, :, :], axis=-1)
    assert d.min() >= 0.1
    r = W.ir_receivers()
    assert np.all(np.abs(r[:, 2] - 1.75) < 1e-12)
    assert np.linalg.norm(r - np.asarray(W.IR_SOURCE), axis=1).min() >= 0.1
    lw = W.cfg_largest(nrec=32)
    assert np.all((lw.receivers > 0.25) & (lw.receivers < np.array(lw.room) - 0.25))
    assert len(set(np.round(lw.beta.real, 12))) == 6   # one admittance per wall
