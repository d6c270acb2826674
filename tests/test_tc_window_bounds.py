"""Host check of the per-item sample-window bound of the tensor-core path.

The kernel bounds every interpolation index k of a (tile, element, transmit)
item by [klo, khi] from per-item quantities alone: the tile's transmit-delay
range plus a receive-offset range, the tangent plane of |p - r| below and
min(tangent + a R^2 / (2 |G|), a R) above (convexity of the distance, and
the triangle inequality).  Here the same bounds are evaluated in float64 and
the exact k of every voxel inside the aperture is checked against them; the
paper's workload and the Table 1 configuration need a single 15-value window
per item, the small test scenes several.
"""
import numpy as np
import pytest

from paper_2606_13259_gb300 import synth as S

KV = 15          # values of k one MMA window covers (16 rows: k and k + 1)
MARGIN = 0.02    # samples


def tile_items(sc, tile):
    """Exact k of the in-aperture voxels of one tile for every (transmit,
    element), and the kernel's [klo, khi] bound for each."""
    a = sc.fs / sc.c
    tx, ty, tz = tile
    ii, jj, kk = np.arange(8) + 8 * tx, np.arange(4) + 4 * ty, np.arange(4) + 4 * tz
    X, Y, Z = np.meshgrid(ii, jj, kk, indexing="ij")
    ok = ((X < sc.nx) & (Y < sc.ny) & (Z < sc.nz)).reshape(-1)
    P = np.stack([sc.origin[0] + sc.spacing[0] * X, sc.origin[1] + sc.spacing[1] * Y,
                  sc.origin[2] + sc.spacing[2] * Z], -1).reshape(-1, 3)
    p0 = np.array([sc.origin[0] + sc.spacing[0] * (8 * tx + 3.5), sc.origin[1] + sc.spacing[1] * (4 * ty + 1.5),
                   sc.origin[2] + sc.spacing[2] * (4 * tz + 1.5)])
    h = np.array([3.5 * sc.spacing[0], 1.5 * sc.spacing[1], 1.5 * sc.spacing[2]])
    R = np.linalg.norm(h)
    pos = sc.elem_pos
    G = p0 - pos
    D0 = np.linalg.norm(G, axis=1)
    R0 = a * D0
    Rb, rf = np.floor(R0), R0 - np.floor(R0)
    lin = np.abs(G / D0[:, None]) @ (a * h)
    lo_off = -lin - MARGIN
    hi_off = np.minimum(lin + a * R * R / (2 * D0), a * R) + MARGIN
    d = P[:, None, :] - pos[None]
    rx = a * np.linalg.norm(d, axis=2) - R0[None]            # receive rest per voxel and element
    inside = (d[..., 2] > 0) & (d[..., 0] ** 2 + d[..., 1] ** 2 <= (1 + 1e-6) * (d[..., 2] / (2 * sc.f_number)) ** 2)
    inside &= ok[:, None]
    out = []
    for q in range(sc.Q):
        if sc.tx_kind[q] == S.TX_PLANE:
            t_all, tc = a * (P @ sc.tx_vec[q]), a * (p0 @ sc.tx_vec[q])
        elif sc.tx_kind[q] == S.TX_NONE:
            t_all, tc = np.zeros(len(P)), 0.0
        else:
            v = sc.tx_vec[q]
            off = np.linalg.norm(v) if sc.t0_offset else 0.0
            t_all, tc = a * (np.linalg.norm(P - v, axis=1) - off), a * (np.linalg.norm(p0 - v) - off)
        tb = np.floor(tc)
        t = t_all - tb
        tmin, tmax = t[ok].min(), t[ok].max()
        k = tb + Rb[None] + np.floor(rf[None] + t[:, None] + rx)
        klo = tb + Rb + np.floor(rf + tmin + lo_off)
        khi = tb + Rb + np.floor(rf + tmax + hi_off)
        out.append((k, inside, klo, khi))
    return out


def check(sc, tiles):
    n_sub = []
    for tile in tiles:
        for k, inside, klo, khi in tile_items(sc, tile):
            for e in np.nonzero(inside.any(0))[0]:
                ke = k[inside[:, e], e]
                assert ke.min() >= klo[e] and ke.max() <= khi[e]
                n_sub.append(int((khi[e] - klo[e]) // KV + 1))
    return np.array(n_sub)


def sample_tiles(sc, n, seed):
    rng = np.random.default_rng(seed)
    nt = ((sc.nx + 7) // 8, (sc.ny + 3) // 4, (sc.nz + 3) // 4)
    return [tuple(int(rng.integers(m)) for m in nt) for _ in range(n)]


@pytest.mark.parametrize("name,n_tiles", [("paper", 12), ("table1", 40)])
def test_full_size_workloads_need_one_window_per_item(name, n_tiles):
    sc = S.scene_paper() if name == "paper" else S.scene_table1()
    ns = check(sc, sample_tiles(sc, n_tiles, seed=5))
    assert ns.size > 0 and ns.max() == 1


def test_small_scene_bounds_hold_with_several_windows():
    sc = S.scene_small_iq()
    nt = ((sc.nx + 7) // 8, (sc.ny + 3) // 4, (sc.nz + 3) // 4)
    tiles = [(x, y, z) for x in range(nt[0]) for y in range(nt[1]) for z in range(nt[2])][::3]
    ns = check(sc, tiles)
    assert ns.max() >= 2
