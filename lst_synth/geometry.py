"""Synthetic detector description: the doublet-module outer tracker the workloads run on.

This module only *describes* the detector (where each module sits).  It holds none of the
tracking method's arithmetic: no cut, window or connection rule lives here.  Both the CPU
oracle and the CUDA library receive the same module table and derive everything else on
their own.

Geometry (cm):
  * 6 barrel doublet layers, lower-sensor radii 23, 36, 51, 68, 86, 110 and sensor gaps
    0.16, 0.16, 0.26, 0.40, 0.40, 0.40; modules are 10 cm in z over |z| < 120 and
    ceil(2*pi*r/10) equal phi sectors.  Layers 1-3 are PS (pixel-strip), 4-6 are 2S (strips).
  * 5 endcap doublet disks per side at |z| = 130, 165, 200, 235, 270 (upper sensor 0.4 cm
    further out in |z|), 9 rings of 10 cm in r in [20, 110), ceil(2*pi*r_mid/10) phi sectors.
    All endcap modules are PS-like (radial coordinate measured to 0.5 mm).

Two features of the Phase-2 layout in the paper's Fig. 1 that the plain geometry leaves
out (Sec. 1) can be switched on: ``realistic=True`` tilts the inner-barrel rows and
``endcap_2s=True`` makes the outer endcap rings 2S modules:
  * tilted inner-barrel modules: in layers 1-3 the rows with |z centre| >= 45 cm are
    tilted towards the interaction point by half the angle under which the row centre is
    seen from it (tilt = atan(|z_c| / r) / 2, sign of z_c).  A tilted module's lower sensor
    is the cone section through (r, z_c) whose normal in the r-z plane is
    (cos tilt, sin tilt), over the same 10 cm z bin; the upper sensor sits one gap along
    that normal;
  * PS and 2S endcap rings: rings at r >= 60 cm are 2S modules (strips: r known only to
    the centre of a 5 cm strip).

The paper describes this structure qualitatively (Sec. 1, Fig. 1: every outer-tracker
layer is two closely spaced sensors; the module is the unit of locality).  The radii,
gaps and extents are the workload recipe's numbers.

The record layout below is the C struct ``lst_module_desc`` (48 bytes); ``tilt`` is the
barrel tilt angle in radians (0: the sensors are the cylinders r = surf, surf + gap).
"""
from __future__ import annotations

import math

import numpy as np

B_FIELD_T = 3.8
# pT [GeV] = PT_PER_CM * R [cm]  (R = pT / (0.3 B) with R in m)
PT_PER_CM = 0.0029979245800 * B_FIELD_T

BARREL_R = (23.0, 36.0, 51.0, 68.0, 86.0, 110.0)
BARREL_GAP = (0.16, 0.16, 0.26, 0.40, 0.40, 0.40)
BARREL_PS = (True, True, True, False, False, False)
BARREL_ZHALF = 120.0
BARREL_ZLEN = 10.0
BARREL_NZ = 24
DISK_Z = (130.0, 165.0, 200.0, 235.0, 270.0)
DISK_GAP = 0.4
RING_R0 = 20.0
RING_DR = 10.0
N_RING = 9
PHI_PITCH = 10.0
TILT_Z = 45.0      # realistic geometry: barrel rows 1-3 with |z centre| >= this are tilted
RING_2S_R = 60.0   # realistic geometry: endcap rings starting at or beyond this radius are 2S

SUBDET_BARREL = 0
SUBDET_ENDCAP = 1
STYPE_PS = 0
STYPE_2S = 1

MODULE_DTYPE = np.dtype(
    [
        ("subdet", np.uint8),
        ("layer", np.uint8),
        ("side", np.int8),
        ("stype", np.uint8),
        ("ieta", np.uint16),
        ("iphi", np.uint16),
        ("nphi", np.uint16),
        ("pad", np.uint16),
        ("surf", np.float32),
        ("gap", np.float32),
        ("emin", np.float32),
        ("emax", np.float32),
        ("e0x", np.float32),
        ("e0y", np.float32),
        ("e1x", np.float32),
        ("e1y", np.float32),
        ("tilt", np.float32),
    ],
    align=False,
)
assert MODULE_DTYPE.itemsize == 48


def _nphi(r: float) -> int:
    return int(math.ceil(2.0 * math.pi * r / PHI_PITCH))


def _edges(n: int) -> np.ndarray:
    """Unit vectors of the n+1 sector edges (edge n is edge 0, bit for bit)."""
    k = np.arange(n, dtype=np.float64)
    ang = 2.0 * np.pi * k / n
    e = np.stack([np.cos(ang), np.sin(ang)], axis=1).astype(np.float32)
    return np.concatenate([e, e[:1]], axis=0)


class Geometry:
    """Module table plus the index helpers the event generator needs.

    ``barrel_only`` drops the endcap disks (the tiny and barrel-batch workloads).
    """

    def __init__(self, barrel_only: bool = False, realistic: bool = False, endcap_2s: bool = False):
        self.barrel_only = barrel_only
        self.realistic = realistic
        self.endcap_2s = endcap_2s
        rows = []
        self.barrel_base = []  # first module id of each barrel layer
        self.barrel_nphi = []
        for li, r in enumerate(BARREL_R):
            n = _nphi(r)
            e = _edges(n)
            self.barrel_base.append(len(rows))
            self.barrel_nphi.append(n)
            for iz in range(BARREL_NZ):
                z0 = -BARREL_ZHALF + iz * BARREL_ZLEN
                zc = z0 + 0.5 * BARREL_ZLEN
                tilt = 0.0
                if realistic and li < 3 and abs(zc) >= TILT_Z:
                    tilt = math.copysign(0.5 * math.atan(abs(zc) / r), zc)
                for k in range(n):
                    rows.append(
                        (SUBDET_BARREL, li + 1, 0, STYPE_PS if BARREL_PS[li] else STYPE_2S,
                         iz, k, n, 0, r, BARREL_GAP[li], z0, z0 + BARREL_ZLEN,
                         e[k, 0], e[k, 1], e[k + 1, 0], e[k + 1, 1], tilt)
                    )
        # endcap_base[(side, disk)][ring] -> first module id of that ring
        self.endcap_base = {}
        self.ring_nphi = [_nphi(RING_R0 + RING_DR * (j + 0.5)) for j in range(N_RING)]
        if not barrel_only:
            ring_edges = [_edges(n) for n in self.ring_nphi]
            for side in (-1, 1):
                for di, zd in enumerate(DISK_Z):
                    bases = []
                    for j in range(N_RING):
                        n = self.ring_nphi[j]
                        e = ring_edges[j]
                        bases.append(len(rows))
                        r0 = RING_R0 + RING_DR * j
                        st = STYPE_2S if endcap_2s and r0 >= RING_2S_R else STYPE_PS
                        for k in range(n):
                            rows.append(
                                (SUBDET_ENDCAP, di + 1, side, st, j, k, n, 0,
                                 side * zd, DISK_GAP, r0, r0 + RING_DR,
                                 e[k, 0], e[k, 1], e[k + 1, 0], e[k + 1, 1], 0.0)
                            )
                    self.endcap_base[(side, di + 1)] = bases
        self.modules = np.array(rows, dtype=MODULE_DTYPE)
        self.n_modules = len(self.modules)
        # (layer, z bin) -> tilt of that barrel row
        self.row_tilt = {}
        for li in range(len(BARREL_R)):
            base = self.barrel_base[li]
            for iz in range(BARREL_NZ):
                self.row_tilt[(li + 1, iz)] = float(self.modules["tilt"][base + iz * self.barrel_nphi[li]])

    # ---- point -> module (used to decide which sensor a simulated particle fired) ----
    def barrel_module(self, layer: np.ndarray, z: np.ndarray, phi: np.ndarray):
        """Module id for points on barrel ``layer`` (1-based); -1 outside |z| < 120."""
        layer = np.asarray(layer)
        iz = np.floor((z + BARREL_ZHALF) / BARREL_ZLEN).astype(np.int64)
        nphi = np.asarray(self.barrel_nphi)[layer - 1]
        base = np.asarray(self.barrel_base)[layer - 1]
        k = np.floor(np.mod(phi, 2 * np.pi) / (2 * np.pi / nphi)).astype(np.int64)
        k = np.minimum(k, nphi - 1)
        ok = (iz >= 0) & (iz < BARREL_NZ)
        return np.where(ok, base + iz * nphi + k, -1)

    def endcap_module(self, side: np.ndarray, disk: np.ndarray, r: np.ndarray, phi: np.ndarray):
        """Module id for points on endcap disk ``disk`` of ``side``; -1 outside the rings."""
        out = np.full(np.shape(r), -1, dtype=np.int64)
        if self.barrel_only:
            return out
        j = np.floor((r - RING_R0) / RING_DR).astype(np.int64)
        ok = (j >= 0) & (j < N_RING)
        jj = np.clip(j, 0, N_RING - 1)
        nphi = np.asarray(self.ring_nphi)[jj]
        k = np.floor(np.mod(phi, 2 * np.pi) / (2 * np.pi / nphi)).astype(np.int64)
        k = np.minimum(k, nphi - 1)
        side = np.broadcast_to(side, np.shape(r))
        disk = np.broadcast_to(disk, np.shape(r))
        for (s, d), bases in self.endcap_base.items():
            sel = ok & (side == s) & (disk == d)
            if np.any(sel):
                b = np.asarray(bases)[jj[sel]]
                out[sel] = b + k[sel]
        return out
