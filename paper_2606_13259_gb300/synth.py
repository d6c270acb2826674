"""Seeded synthetic inputs: imaging scenes and simulated channel data.

This module describes the acquisition (array, grid, transmits) and simulates
what the array records from a set of point reflectors.  It holds none of the
beamforming arithmetic: no voxel-to-element delays, no interpolation, no sums
over channels.  It is shared by the tests, the benchmark and users who want a
phantom; it imports neither the CUDA binding nor the CPU oracle.

Scenes follow the workloads of the paper's evaluation (Sec. 4, Table 1): a
matrix array of M elements, a voxel grid of N voxels, Q diverging-wave
transmits, channel data y[b][q][m][k] (Sec. 2, batched layout with samples
contiguous).  The paper simulates reflectors on a trefoil knot in the frequency
domain (Sec. 4, "Synthetic data generation") and notes that performance does
not depend on the data; here reflectors are uniform speckle plus a few bright
points, simulated in the time domain with a Gaussian-modulated pulse.

Random numbers come from numpy's PCG64 generator seeded per frame; the pulse
splatting runs in torch on any device.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

TX_DIVERGING = 0
TX_PLANE = 1
TX_NONE = 2

MM = 1e-3


@dataclasses.dataclass
class Scene:
    """Geometry and acquisition parameters of one beamforming plan.

    Voxel (ix, iy, iz) sits at origin + spacing * (ix, iy, iz); images are
    stored [iz][iy][ix] (x fastest).  Channel data are [b][q][m][k].
    """

    name: str
    nx: int
    ny: int
    nz: int
    origin: tuple
    spacing: tuple
    elem_pos: np.ndarray          # (M, 3) metres
    elem_normal: np.ndarray       # (M, 3) unit vectors
    tx_kind: np.ndarray           # (Q,) int32, TX_*
    tx_vec: np.ndarray            # (Q, 3) virtual source (m) or unit direction
    t0_ref: tuple = (0.0, 0.0, 0.0)
    t0_offset: bool = True
    c: float = 1540.0
    fs: float = 30e6
    f_demod: float = 0.0
    f_number: float = 1.0
    K: int = 512
    iq: bool = False
    fc: float = 7.5e6
    w_tx: Optional[np.ndarray] = None   # (Q, N) float32 or None

    @property
    def M(self) -> int:
        return int(self.elem_pos.shape[0])

    @property
    def Q(self) -> int:
        return int(self.tx_vec.shape[0])

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def with_(self, **kw) -> "Scene":
        return dataclasses.replace(self, **kw)

    def voxel_index(self, ix: int, iy: int, iz: int) -> int:
        return (iz * self.ny + iy) * self.nx + ix

    def voxel_centre(self, ix: int, iy: int, iz: int) -> np.ndarray:
        return np.array(self.origin) + np.array(self.spacing) * np.array([ix, iy, iz], dtype=np.float64)

    def describe(self) -> dict:
        return {
            "name": self.name, "grid": [self.nx, self.ny, self.nz],
            "spacing_mm": [s / MM for s in self.spacing], "M": self.M, "Q": self.Q,
            "K": self.K, "iq": self.iq, "c": self.c, "fs": self.fs,
            "f_demod": self.f_demod, "f_number": self.f_number,
        }


def matrix_array(n_x: int, n_y: int, pitch: float) -> tuple[np.ndarray, np.ndarray]:
    """Flat matrix array centred on the origin, normals +z; element m = j_y * n_x + j_x."""
    jx, jy = np.meshgrid(np.arange(n_x), np.arange(n_y), indexing="xy")
    pos = np.zeros((n_x * n_y, 3))
    pos[:, 0] = (jx.ravel() - (n_x - 1) / 2.0) * pitch
    pos[:, 1] = (jy.ravel() - (n_y - 1) / 2.0) * pitch
    nrm = np.zeros_like(pos)
    nrm[:, 2] = 1.0
    return pos, nrm


def source_lattice(xs: Sequence[float], ys: Sequence[float], z: float) -> np.ndarray:
    """Virtual sources on a lattice behind the array (one per (x, y) pair, x fastest)."""
    return np.array([[x, y, z] for y in ys for x in xs], dtype=np.float64)


def centred_origin(nx: int, ny: int, dx: float, dy: float, z0: float) -> tuple:
    return (-(nx - 1) / 2.0 * dx, -(ny - 1) / 2.0 * dy, z0)


def _diverging(vs: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    return np.full(len(vs), TX_DIVERGING, dtype=np.int32), np.asarray(vs, dtype=np.float64)


# --------------------------------------------------------------------------
# The workloads
# --------------------------------------------------------------------------

def scene_small() -> Scene:
    """32^3 voxels at 0.2 mm (depth 5 to 11.2 mm), 16x16 elements at 0.3 mm,
    one diverging wave from 10 mm behind the array, fc 7.5 MHz, fs 30 MHz,
    512 real RF samples, f-number 1."""
    pos, nrm = matrix_array(16, 16, 0.3 * MM)
    kind, vec = _diverging([[0.0, 0.0, -10 * MM]])
    return Scene("small_rf_32cube_256el_1tx", 32, 32, 32, centred_origin(32, 32, 0.2 * MM, 0.2 * MM, 5 * MM),
                 (0.2 * MM,) * 3, pos, nrm, kind, vec, c=1540.0, fs=30e6, f_demod=0.0,
                 f_number=1.0, K=512, iq=False, fc=7.5e6)


def scene_paper(K: int = 2048) -> Scene:
    """Paper-scale problem (Sec. 2: N = 128^3, M = 32^2, Q = 16): 0.1 mm voxels
    from 5 mm depth, 32x32 elements at 0.3 mm, 16 virtual sources on a 4x4
    lattice (3 mm pitch) 10 mm behind the array, complex IQ demodulated at
    fc = 7.5 MHz and sampled at fs = 15 MHz, K samples."""
    pos, nrm = matrix_array(32, 32, 0.3 * MM)
    lat = [-4.5 * MM, -1.5 * MM, 1.5 * MM, 4.5 * MM]
    kind, vec = _diverging(source_lattice(lat, lat, -10 * MM))
    return Scene("paper_iq_128cube_1024el_16tx", 128, 128, 128,
                 centred_origin(128, 128, 0.1 * MM, 0.1 * MM, 5 * MM), (0.1 * MM,) * 3,
                 pos, nrm, kind, vec, c=1540.0, fs=15e6, f_demod=7.5e6, f_number=1.0,
                 K=K, iq=True, fc=7.5e6)


def scene_small_iq() -> Scene:
    """The small problem with complex IQ data (demodulated at fc, same fs and K)."""
    return scene_small().with_(name="small_iq_32cube_256el_1tx", iq=True, f_demod=7.5e6)


def scene_diff(c: float = 1540.0) -> Scene:
    """96^3 voxels at 0.1 mm from 5 mm, 32x32 elements, 8 virtual sources on a
    4x2 lattice, IQ, 1536 samples; beamforming sound speed c."""
    pos, nrm = matrix_array(32, 32, 0.3 * MM)
    kind, vec = _diverging(source_lattice([-4.5 * MM, -1.5 * MM, 1.5 * MM, 4.5 * MM],
                                          [-1.5 * MM, 1.5 * MM], -10 * MM))
    return Scene("diff_iq_96cube_1024el_8tx", 96, 96, 96, centred_origin(96, 96, 0.1 * MM, 0.1 * MM, 5 * MM),
                 (0.1 * MM,) * 3, pos, nrm, kind, vec, c=c, fs=15e6, f_demod=7.5e6, f_number=1.0,
                 K=1536, iq=True, fc=7.5e6)


def scenes_batched() -> list[Scene]:
    """Three uneven plans: 64^3 / 16x32 el / 4 tx / K 1024; 96(z)x128x128 /
    1024 el / 9 tx / K 1536; 128^3 / 1024 el / 16 tx / K 2048.  IQ at 15 MHz."""
    pos1, nrm1 = matrix_array(16, 32, 0.3 * MM)
    k1, v1 = _diverging(source_lattice([-1.5 * MM, 1.5 * MM], [-1.5 * MM, 1.5 * MM], -10 * MM))
    p1 = Scene("batched_p1_64cube_512el_4tx", 64, 64, 64, centred_origin(64, 64, 0.1 * MM, 0.1 * MM, 5 * MM),
               (0.1 * MM,) * 3, pos1, nrm1, k1, v1, c=1540.0, fs=15e6, f_demod=7.5e6,
               f_number=1.0, K=1024, iq=True, fc=7.5e6)
    pos2, nrm2 = matrix_array(32, 32, 0.3 * MM)
    k2, v2 = _diverging(source_lattice([-3 * MM, 0.0, 3 * MM], [-3 * MM, 0.0, 3 * MM], -10 * MM))
    p2 = Scene("batched_p2_128x128x96_1024el_9tx", 128, 128, 96,
               centred_origin(128, 128, 0.1 * MM, 0.1 * MM, 5 * MM), (0.1 * MM,) * 3, pos2, nrm2,
               k2, v2, c=1540.0, fs=15e6, f_demod=7.5e6, f_number=1.0, K=1536, iq=True, fc=7.5e6)
    p3 = scene_paper(2048).with_(name="batched_p3_128cube_1024el_16tx")
    return [p1, p2, p3]


def scene_table1(fc: float = 7.5e6, c: float = 1540.0) -> Scene:
    """The evaluation configuration of the paper's Table 1: M = 32 x 32
    elements at a pitch of one wavelength, N = 128^3 voxels at half a
    wavelength, Q = 1 observation, K = 256 samples.  The table leaves the
    transmit, the sampling rate and the depth open; here one plane wave at
    normal incidence, IQ sampled at 2 fc (K = 256 then spans 128 wavelengths
    of two-way path, the depth extent of the grid), first voxel half a
    wavelength below the array, f-number 1."""
    lam = c / fc
    pos, nrm = matrix_array(32, 32, lam)
    kind = np.array([TX_PLANE], dtype=np.int32)
    vec = np.array([[0.0, 0.0, 1.0]])
    return Scene("table1_iq_128cube_1024el_1tx", 128, 128, 128, centred_origin(128, 128, lam / 2, lam / 2, lam / 2),
                 (lam / 2,) * 3, pos, nrm, kind, vec, c=c, fs=2 * fc, f_demod=fc, f_number=1.0, K=256, iq=True,
                 fc=fc)


def scene_tiny(iq: bool = True, n: tuple = (3, 3, 3), elems: tuple = (2, 2), n_tx: int = 2,
               K: int = 64, f_number: float = 0.0) -> Scene:
    """A few voxels and elements for brute-force checks (fs 30 MHz, 0.1 mm voxels from 1 mm depth)."""
    pos, nrm = matrix_array(elems[0], elems[1], 0.3 * MM)
    src = [[0.4 * MM * (q - (n_tx - 1) / 2.0), 0.0, -5 * MM] for q in range(n_tx)]
    kind, vec = _diverging(src)
    return Scene("tiny", n[0], n[1], n[2], centred_origin(n[0], n[1], 0.1 * MM, 0.1 * MM, 1.0 * MM),
                 (0.1 * MM,) * 3, pos, nrm, kind, vec, c=1540.0, fs=30e6,
                 f_demod=7.5e6 if iq else 0.0, f_number=f_number, K=K, iq=iq, fc=7.5e6)


# --------------------------------------------------------------------------
# Phantoms and the acquisition simulator
# --------------------------------------------------------------------------

SMALL_POINTS = [(10, 16, 8), (16, 16, 16), (22, 12, 24)]


def paper_points(scene: Scene) -> list[tuple[int, int, int]]:
    """Ten bright points at voxel centres spread through the volume."""
    f = [(0.5, 0.5, 0.25), (0.3, 0.6, 0.4), (0.7, 0.4, 0.4), (0.5, 0.5, 0.5), (0.25, 0.25, 0.6),
         (0.75, 0.75, 0.6), (0.4, 0.7, 0.75), (0.6, 0.3, 0.75), (0.5, 0.5, 0.85), (0.35, 0.45, 0.9)]
    return [(int(a * (scene.nx - 1)), int(b * (scene.ny - 1)), int(c * (scene.nz - 1))) for a, b, c in f]


def phantom(scene: Scene, n_speckle: int, points: Sequence[tuple], seed: int,
            point_amp: float = 50.0) -> tuple[np.ndarray, np.ndarray]:
    """Speckle reflectors uniform in the grid box with N(0, 1) amplitudes, plus
    bright points (amplitude point_amp) at the given voxel centres."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array(scene.origin)
    hi = lo + np.array(scene.spacing) * (np.array([scene.nx, scene.ny, scene.nz]) - 1)
    pos = lo + (hi - lo) * rng.random((n_speckle, 3))
    amp = rng.standard_normal(n_speckle)
    if points:
        pts = np.array([scene.voxel_centre(*p) for p in points])
        pos = np.concatenate([pos, pts])
        amp = np.concatenate([amp, np.full(len(points), point_amp)])
    return pos, amp


def arrival_times(scene: Scene, pos, c: float):
    """Two-way travel time (seconds) from transmit to reflector to element,
    [Q][M][L], for reflectors pos (L, 3) (a torch tensor).  The clock starts
    when the transmitted wave passes t0_ref (for a diverging wave:
    ||s - v|| - ||v - t0_ref||); plane waves start at t0_ref; without a
    transmit only the return path counts."""
    import torch

    s = pos                                      # (L, 3)
    as_t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=s.dtype, device=s.device)
    r = as_t(scene.elem_pos)
    back = torch.sqrt(((s[None, :, :] - r[:, None, :]) ** 2).sum(-1))     # (M, L)
    t0 = as_t(scene.t0_ref)
    outs = []
    for q in range(scene.Q):
        v = as_t(scene.tx_vec[q])
        kind = int(scene.tx_kind[q])
        if kind == TX_DIVERGING:
            out_path = torch.sqrt(((s - v) ** 2).sum(-1))
            if scene.t0_offset:
                out_path = out_path - float(np.linalg.norm(scene.tx_vec[q] - np.asarray(scene.t0_ref)))
        elif kind == TX_PLANE:
            out_path = ((s - t0) * v).sum(-1)
        else:
            out_path = torch.zeros(s.shape[0], dtype=s.dtype, device=s.device)
        outs.append((out_path[None, :] + back) / c)
    return torch.stack(outs)                     # (Q, M, L)


def simulate(scene: Scene, pos: np.ndarray, amp: np.ndarray, *, c: Optional[float] = None,
             noise_db: Optional[float] = None, seed: int = 0, device="cpu", chunk: int = 512):
    """Channel data of one acquisition, torch tensor [Q][M][K] (complex64 for IQ,
    float32 for RF) on `device`.

    RF echo of a reflector with amplitude a arriving at tau:
        a * g(t - tau) * cos(2 pi fc (t - tau)),  g(t) = exp(-t^2 / (2 sigma^2)),
    with an envelope full width at half maximum of two periods.  IQ data are
    the complex baseband of that echo after demodulation at f_demod:
        a * g(t - tau) * exp(i 2 pi (fc - f_demod) (t - tau)) * exp(-i 2 pi f_demod tau).
    Samples sit at t = k / fs.  White Gaussian noise noise_db below the RMS of
    the echoes is added when noise_db is given.
    """
    import torch

    c = scene.c if c is None else c
    dev = torch.device(device)
    K, Q, M = scene.K, scene.Q, scene.M
    sigma_s = (2.0 / scene.fc) / (2.0 * math.sqrt(2.0 * math.log(2.0))) * scene.fs   # envelope width, samples
    half = int(math.ceil(4.0 * sigma_s)) + 1
    taps = torch.arange(-half, half + 2, device=dev, dtype=torch.float32)        # (T,)
    out = torch.zeros(Q * M * K, 2, device=dev, dtype=torch.float32)
    row = (torch.arange(Q * M, device=dev, dtype=torch.int64) * K).view(Q, M, 1, 1)
    pos_t = torch.as_tensor(pos, dtype=torch.float64, device=dev)
    amp_t = torch.as_tensor(amp, dtype=torch.float32, device=dev)
    w_env = 1.0 / (2.0 * sigma_s * sigma_s)
    w_bb = 2.0 * math.pi * (scene.fc - scene.f_demod) / scene.fs                  # baseband rad/sample
    for s0 in range(0, pos_t.shape[0], chunk):
        tau = arrival_times(scene, pos_t[s0:s0 + chunk], c)                     # (Q, M, L) s, float64
        ts = tau * scene.fs
        k0 = torch.floor(ts)
        frac = (ts - k0).to(torch.float32).unsqueeze(-1)                         # (Q, M, L, 1)
        dts = taps - frac                                                        # t - tau, samples
        env = amp_t[s0:s0 + chunk].view(1, 1, -1, 1) * torch.exp(-dts * dts * w_env)
        kk = k0.to(torch.int64).unsqueeze(-1) + taps.to(torch.int64)
        valid = (kk >= 0) & (kk <= K - 1)
        if scene.iq:
            # exp(-i 2 pi f_d tau) reduced to one turn in float64, then float32
            turns = tau * scene.f_demod
            carrier = (2.0 * math.pi * (turns - torch.floor(turns))).to(torch.float32).unsqueeze(-1)
            ph = w_bb * dts - carrier
            vals = torch.stack([env * torch.cos(ph), env * torch.sin(ph)], -1)
        else:
            ph = (2.0 * math.pi * scene.fc / scene.fs) * dts
            vals = torch.stack([env * torch.cos(ph), torch.zeros_like(env)], -1)
        idx = (row + kk.clamp(0, K - 1)).reshape(-1)
        vals = (vals * valid.unsqueeze(-1)).reshape(-1, 2)
        out.index_add_(0, idx, vals)
    if noise_db is not None:
        rng = np.random.Generator(np.random.PCG64(seed + 7919))
        ncomp = 2 if scene.iq else 1
        sig_rms = float(torch.sqrt((out[:, :ncomp].double() ** 2).sum(-1).mean()))
        nz = rng.standard_normal((Q * M * K, ncomp)).astype(np.float32)
        scale = sig_rms * 10 ** (-noise_db / 20.0) / math.sqrt(ncomp)
        out[:, :ncomp] += torch.as_tensor(nz, device=dev) * scale
    if scene.iq:
        return torch.view_as_complex(out.contiguous()).view(Q, M, K)
    return out[:, 0].contiguous().view(Q, M, K)


def frames(scene: Scene, n_frames: int, seed: int, n_speckle: int, points, *, noise_db=None,
           c: Optional[float] = None, device="cpu"):
    """n_frames independent acquisitions [B][Q][M][K]; frame f uses seed + f."""
    import torch

    out = []
    for f in range(n_frames):
        pos, amp = phantom(scene, n_speckle, points, seed + 1000 * f)
        out.append(simulate(scene, pos, amp, c=c, noise_db=noise_db, seed=seed + 1000 * f, device=device))
    return torch.stack(out)


def random_channels(scene: Scene, B: int, seed: int, device="cpu"):
    """Seeded white Gaussian channel data [B][Q][M][K] (complex64 or float32)."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (B, scene.Q, scene.M, scene.K)
    if scene.iq:
        a = rng.standard_normal(shape + (2,)).astype(np.float32)
        return torch.view_as_complex(torch.as_tensor(a)).to(device)
    return torch.as_tensor(rng.standard_normal(shape).astype(np.float32)).to(device)


def random_image(scene: Scene, B: int, seed: int, device="cpu"):
    """Seeded complex Gaussian image-space array [B][N] (complex64)."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((B, scene.N, 2)).astype(np.float32)
    return torch.view_as_complex(torch.as_tensor(a)).to(device)
