"""Seeded synthetic inputs for the SVT linearised track fit.

This module only MAKES inputs: packed event words (event / road / hit words),
the int16 fit-constant table and FP32 calibration tracks.  It never applies
fit constants to coordinates, never forms a combination and never computes a
chi-square, so it holds none of the method's arithmetic.  Both the CUDA path
and the CPU oracle consume what it produces.

Physics recipe (the paper, Sec. 2: hits are fitted with a linear form
``p = f.x + q`` whose constants are pre-computed; Sec. 4: events carry a fixed
number of combinations and batches run from 1 to 3000 events):

* A track has impact parameter ``d0`` (cm), azimuth ``phi0`` and half-curvature
  ``c = rho/2`` (1/cm, ``rho = 0.003 B / pT`` with B = 1.4 T).
* Coordinates 0..4 are the azimuth measured at radii 2.5, 4.1, 6.5, 10.6 cm
  (silicon-like) and 106 cm (track-trigger phi); coordinate 5 is the
  track-trigger curvature.  Each is quantised to an unsigned 15-bit local
  coordinate inside the road's azimuthal sector.
* ``linear`` mode uses the first-order form ``phi(r) = phi0 + d0/r + c r``;
  ``helix`` mode uses the exact circle.
* Each sector has its own small misalignment (radius scale and offsets), so the
  constants differ between sectors.
* Fit constants per (sector, layer mask): parameter rows are the weighted
  least-squares estimator ``(A^T W A)^-1 A^T W`` of the linear model
  ``x = x0 + A theta``; the three chi rows are an orthonormal basis of the null
  space of the whitened design matrix, so for true hits each chi component is
  a unit Gaussian before scaling.  Rows are scaled to int16 with round-half-even.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# --- packed word format ------------------------------------------------------
# type in bits [31:30]: 3 = event header, 2 = road header, 0 = hit, 1 = invalid.
# event header: [29:12] event id, [11:0] number of roads
# road header : [29:21] sector,   [20:0] road id
# hit         : [29:27] layer,    [26:15] reserved (0), [14:0] coordinate
TYPE_HIT, TYPE_ROAD, TYPE_EVENT = 0, 2, 3
N_LAYERS = 6
N_MASKS = 64
COORD_MAX = 32767
MAX_HITS_PER_LAYER = 16
MAX_ROADS_PER_EVENT = 4095
MAX_SECTORS = 512


def event_word(event_id, n_roads):
    return ((np.uint32(TYPE_EVENT) << np.uint32(30))
            | ((np.asarray(event_id, np.uint32) & np.uint32(0x3FFFF)) << np.uint32(12))
            | (np.asarray(n_roads, np.uint32) & np.uint32(0xFFF)))


def road_word(sector, road_id):
    return ((np.uint32(TYPE_ROAD) << np.uint32(30))
            | ((np.asarray(sector, np.uint32) & np.uint32(0x1FF)) << np.uint32(21))
            | (np.asarray(road_id, np.uint32) & np.uint32(0x1FFFFF)))


def hit_word(layer, coord):
    return (((np.asarray(layer, np.uint32) & np.uint32(7)) << np.uint32(27))
            | (np.asarray(coord, np.uint32) & np.uint32(0x7FFF)))


# --- geometry ----------------------------------------------------------------
RADII_CM = np.array([2.5, 4.1, 6.5, 10.6, 106.0])
B_TESLA = 1.4
PT_MIN, PT_MAX = 2.0, 20.0
D0_MAX_CM = 0.1
C_MAX = 0.003 * B_TESLA / PT_MIN / 2.0          # largest half-curvature, 1/cm
SIGMA_LSB = np.array([180.0, 130.0, 100.0, 80.0, 240.0, 160.0])
F_LIMIT = 30000.0                                # largest |int16| a scaled row may use
CHI2_Q99_3DOF = 11.344866730144373              # 99th percentile of chi-square, 3 dof
BASE_SEED = 20131101


@dataclass
class Geometry:
    n_sectors: int
    radius: np.ndarray        # [S, 5] misaligned radii (cm)
    offset: np.ndarray        # [S, 6] phi offsets (rad) for l<5, curvature offset for l=5
    window: np.ndarray        # [5] full azimuthal window per phi layer (rad)

    @property
    def sector_width(self):
        return 2.0 * np.pi / self.n_sectors

    def centre(self, sector):
        return (np.asarray(sector, np.float64) + 0.5) * self.sector_width

    def lsb_scale(self):
        """LSB per physical unit for every coordinate: [6]."""
        s = np.empty(6)
        s[:5] = 32768.0 / self.window
        s[5] = 16384.0 / C_MAX
        return s


def make_geometry(n_sectors: int, seed: int) -> Geometry:
    rng = np.random.default_rng([seed, 0xC0])
    width = 2.0 * np.pi / n_sectors
    half = 1.15 * (width / 2 + D0_MAX_CM / RADII_CM + C_MAX * RADII_CM)
    window = 2.0 * half
    radius = RADII_CM[None, :] * (1.0 + rng.normal(0.0, 2e-3, size=(n_sectors, 5)))
    lsb_rad = window / 32768.0
    offset = np.empty((n_sectors, 6))
    offset[:, :5] = rng.normal(0.0, 20.0, size=(n_sectors, 5)) * lsb_rad[None, :]
    offset[:, 5] = rng.normal(0.0, 20.0, size=n_sectors) * (C_MAX / 16384.0)
    return Geometry(n_sectors, radius, offset, window)


def design(geo: Geometry, sector):
    """Linear model of the coordinates: x = x0 + A @ (d0, dphi0, c).

    dphi0 is the azimuth relative to the sector centre.  Returns (A [.,6,3],
    x0 [.,6]) in LSB per physical unit and LSB.
    """
    sector = np.atleast_1d(np.asarray(sector))
    r = geo.radius[sector]                       # [n,5]
    scale = geo.lsb_scale()
    A = np.zeros((len(sector), 6, 3))
    A[:, :5, 0] = scale[None, :5] / r
    A[:, :5, 1] = scale[None, :5]
    A[:, :5, 2] = scale[None, :5] * r
    A[:, 5, 2] = scale[5]
    x0 = 16384.0 - geo.offset[sector] * scale[None, :]
    return A, x0


def true_coords(geo: Geometry, sector, d0, phi0, c, mode="helix"):
    """Unquantised coordinates (LSB, float) of tracks: [n, 6]."""
    sector = np.asarray(sector)
    r = geo.radius[sector]                       # [n,5]
    d0 = np.asarray(d0, np.float64)[:, None]
    cc = np.asarray(c, np.float64)[:, None]
    dphi0 = (np.asarray(phi0, np.float64) - geo.centre(sector))[:, None]
    if mode == "linear":
        phi_rel = dphi0 + d0 / r + cc * r
    elif mode == "helix":
        rho = 2.0 * cc
        arg = (rho * (r * r + d0 * d0) / 2.0 + d0) / (r * (1.0 + rho * d0))
        phi_rel = dphi0 + np.arcsin(np.clip(arg, -1.0, 1.0))
    else:
        raise ValueError(mode)
    scale = geo.lsb_scale()
    x = np.empty((len(sector), 6))
    x[:, :5] = 16384.0 + (phi_rel - geo.offset[sector, :5]) * scale[None, :5]
    x[:, 5] = 16384.0 + (cc[:, 0] - geo.offset[sector, 5]) * scale[5]
    return x


# --- fit constants -----------------------------------------------------------
@dataclass
class Constants:
    F: np.ndarray              # int16 [S, 64, 6, 6]  F[s][m][k][l]
    q: np.ndarray              # int16 [S, 64, 6]
    oshift: int
    qshift: int
    unit: np.ndarray           # [3] physical size of one output LSB of d0 (cm), dphi0 (rad), c (1/cm)
    unit_chi: float            # one chi LSB in units of the hit resolution
    chi2_cut_99: int           # 99 % of true-track chi2 under Gaussian smearing
    geometry: Geometry = field(repr=False)

    @property
    def n_sectors(self):
        return self.F.shape[0]


def _mask_layers(m):
    return [l for l in range(N_LAYERS) if (m >> l) & 1]


def make_constants(n_sectors: int, seed: int = BASE_SEED, oshift: int = 15,
                   qshift: int = 15, sigma=SIGMA_LSB, min_fit_layers: int = 5) -> Constants:
    """Fit constants for every sector and every layer mask with at least
    ``min_fit_layers`` (>= 3) layers; rows of the other masks stay zero."""
    geo = make_geometry(n_sectors, seed)
    sectors = np.arange(n_sectors)
    A_all, x0_all = design(geo, sectors)
    sigma = np.asarray(sigma, np.float64)
    par = np.zeros((n_sectors, N_MASKS, 3, 6))
    par_q = np.zeros((n_sectors, N_MASKS, 3))
    chi = np.zeros((n_sectors, N_MASKS, 3, 6))
    chi_q = np.zeros((n_sectors, N_MASKS, 3))
    for m in range(N_MASKS):
        lay = _mask_layers(m)
        n = len(lay)
        if n < max(3, min_fit_layers):
            continue
        A = A_all[:, lay, :]                       # [S,n,3]
        x0 = x0_all[:, lay]                        # [S,n]
        w = 1.0 / sigma[lay] ** 2
        AtW = np.transpose(A, (0, 2, 1)) * w[None, None, :]
        est = np.linalg.solve(AtW @ A, AtW)        # [S,3,n]
        par[:, m][:, :, lay] = est
        par_q[:, m] = -np.einsum("skn,sn->sk", est, x0)
        if n > 3:
            Aw = A / sigma[lay][None, :, None]
            Q, _ = np.linalg.qr(Aw, mode="complete")  # [S,n,n]
            N = Q[:, :, 3:]                            # [S,n,n-3]
            rows = np.transpose(N, (0, 2, 1)) / sigma[lay][None, None, :]
            chi[:, m, : n - 3][:, :, lay] = rows
            chi_q[:, m, : n - 3] = -np.einsum("skn,sn->sk", rows, x0)
    two_o = float(2 ** oshift)
    two_oq = float(2 ** (oshift - qshift)) if oshift >= qshift else 1.0 / float(2 ** (qshift - oshift))
    unit = np.empty(3)
    for k in range(3):
        unit[k] = max(np.abs(par[:, :, k]).max() * two_o / F_LIMIT,
                      np.abs(par_q[:, :, k]).max() * two_oq / F_LIMIT)
    unit_chi = max(np.abs(chi).max() * two_o / F_LIMIT, np.abs(chi_q).max() * two_oq / F_LIMIT)
    F = np.zeros((n_sectors, N_MASKS, 6, 6), np.int16)
    q = np.zeros((n_sectors, N_MASKS, 6), np.int16)
    F[:, :, :3, :] = np.rint(par * two_o / unit[None, None, :, None]).astype(np.int16)
    q[:, :, :3] = np.rint(par_q * two_oq / unit[None, None, :]).astype(np.int16)
    F[:, :, 3:, :] = np.rint(chi * two_o / unit_chi).astype(np.int16)
    q[:, :, 3:] = np.rint(chi_q * two_oq / unit_chi).astype(np.int16)
    cut = int(round(CHI2_Q99_3DOF / unit_chi ** 2))
    return Constants(F, q, oshift, qshift, unit, unit_chi, cut, geo)


# --- batch specs -------------------------------------------------------------
@dataclass(frozen=True)
class BatchSpec:
    """Shape of a synthetic batch."""
    name: str
    n_sectors: int
    roads: tuple               # ("const", n) | ("poisson", mean) | ("loguniform", max)
    hits: tuple                # ("const", n) | ("uniform", lo, hi) | ("geom_cap", p, cap)
    max_comb: int
    seed: int
    noise: float = 0.2
    mode: str = "helix"
    xft: bool = False          # layers 4, 5 come in pairs from one track-trigger track

    def sample_roads(self, rng, n):
        kind = self.roads[0]
        if kind == "const":
            return np.full(n, self.roads[1], np.int64)
        if kind == "poisson":
            return np.minimum(rng.poisson(self.roads[1], n), MAX_ROADS_PER_EVENT).astype(np.int64)
        if kind == "loguniform":
            hi = self.roads[1]
            v = np.floor(np.exp(rng.uniform(0.0, np.log(hi + 1.0), n)))
            return np.clip(v, 1, hi).astype(np.int64)
        raise ValueError(kind)

    def sample_hits(self, rng, n_roads):
        kind = self.hits[0]
        shape = (n_roads, N_LAYERS)
        if kind == "const":
            return np.full(shape, self.hits[1], np.int64)
        if kind == "uniform":
            return rng.integers(self.hits[1], self.hits[2] + 1, size=shape).astype(np.int64)
        if kind == "geom_cap":
            return np.minimum(rng.geometric(self.hits[1], size=shape), self.hits[2]).astype(np.int64)
        raise ValueError(kind)


SPECS = {
    # 100 events x 16 roads, 1-2 hits per layer, 64 sectors
    "small": BatchSpec("small", 64, ("const", 16), ("uniform", 1, 2), 64, BASE_SEED + 0),
    # roads Poisson(64), hits geometric mean 3 capped at 8, 512 sectors, uncapped
    "scaled": BatchSpec("scaled", 512, ("poisson", 64), ("geom_cap", 1.0 / 3.0, 8), 262144, BASE_SEED + 1),
    # roads log-uniform in 1..2048, 1-16 hits per layer, 4096 combinations per road at most
    "uneven": BatchSpec("uneven", 512, ("loguniform", 2048), ("uniform", 1, 16), 4096, BASE_SEED + 2),
    # the paper's fixed shape: 2048 combinations per event = 32 roads x 2^6
    "paper": BatchSpec("paper", 512, ("const", 32), ("const", 2), 262144, BASE_SEED + 5),
    # the scaled shape with layers 4 and 5 paired (one track-trigger track per pair)
    "xft": BatchSpec("xft", 512, ("poisson", 64), ("geom_cap", 1.0 / 3.0, 8), 262144,
                     BASE_SEED + 6, xft=True),
}


@dataclass
class Batch:
    words: np.ndarray          # uint32 [n_words]
    event_off: np.ndarray      # uint64 [n_events + 1]
    n_roads: np.ndarray        # int64  [n_events]
    n_hits: np.ndarray         # int64  [R, 6]
    sector: np.ndarray         # int64  [R]
    d0: np.ndarray             # [R] truth per road
    phi0: np.ndarray
    c: np.ndarray
    xft: bool = False          # layers 4, 5 paired

    @property
    def n_events(self):
        return len(self.n_roads)

    @property
    def total_roads(self):
        return int(self.n_roads.sum())

    def combinations(self, max_comb=None):
        """Combinations per road, prod(max(n_l,1)) (layer 5 left out when it is
        paired with layer 4), optionally capped."""
        n = np.maximum(self.n_hits, 1)
        cnt = np.prod(n[:, :5] if self.xft else n, axis=1)
        return cnt if max_comb is None else np.minimum(cnt, max_comb)


def _gen_chunk(spec, consts, rng, n_events, first_event, first_road):
    geo = consts.geometry
    S = consts.n_sectors
    n_roads = spec.sample_roads(rng, n_events)
    R = int(n_roads.sum())
    n_hits = spec.sample_hits(rng, R)
    if spec.xft:
        n_hits[:, 5] = n_hits[:, 4]
    d0 = rng.uniform(-D0_MAX_CM, D0_MAX_CM, R)
    phi0 = rng.uniform(0.0, 2.0 * np.pi, R)
    pt = rng.uniform(PT_MIN, PT_MAX, R)
    charge = np.where(rng.random(R) < 0.5, -1.0, 1.0)
    c = charge * 0.003 * B_TESLA / pt / 2.0
    sector = np.minimum((phi0 / (2.0 * np.pi / S)).astype(np.int64), S - 1)
    xt = true_coords(geo, sector, d0, phi0, c, spec.mode)       # [R,6]

    per_road = n_hits.sum(axis=1)                                 # [R]
    H = int(per_road.sum())
    flat_counts = n_hits.ravel()
    grp = np.repeat(np.arange(R * N_LAYERS), flat_counts)         # (road, layer) of each hit
    road_of_hit = grp // N_LAYERS
    layer_of_hit = grp % N_LAYERS
    noise = rng.random(H) < spec.noise
    if spec.xft:
        # hit i of layer 5 is the second coordinate of the track of hit i of
        # layer 4: both are the road's track or both are a fake track
        l5 = np.nonzero(layer_of_hit == 5)[0]
        noise[l5] = noise[l5 - n_hits[road_of_hit[l5], 4]]
    smear = rng.normal(0.0, 1.0, H) * SIGMA_LSB[layer_of_hit]
    coord = np.rint(xt[road_of_hit, layer_of_hit] + smear)
    coord = np.where(noise, rng.integers(0, COORD_MAX + 1, H), coord)
    coord = np.clip(coord, 0, COORD_MAX).astype(np.uint32)

    ev_of_road = np.repeat(np.arange(n_events), n_roads)
    ev_len = 1 + np.bincount(ev_of_road, weights=1 + per_road, minlength=n_events).astype(np.int64)
    event_off = np.zeros(n_events + 1, np.int64)
    np.cumsum(ev_len, out=event_off[1:])
    n_words = int(event_off[-1])
    road_len = 1 + per_road
    road_cum = np.zeros(R + 1, np.int64)
    np.cumsum(road_len, out=road_cum[1:])
    road_pos = road_cum[:-1] + ev_of_road + 1                    # header word of each road
    hit_start = np.zeros(R + 1, np.int64)
    np.cumsum(per_road, out=hit_start[1:])
    rank = np.arange(H) - hit_start[road_of_hit]
    hit_pos = road_pos[road_of_hit] + 1 + rank

    words = np.empty(n_words, np.uint32)
    ev_ids = (first_event + np.arange(n_events)) & 0x3FFFF
    words[event_off[:-1]] = event_word(ev_ids, n_roads)
    words[road_pos] = road_word(sector, (first_road + np.arange(R)) & 0x1FFFFF)
    words[hit_pos] = hit_word(layer_of_hit, coord)
    return words, event_off, n_roads, n_hits, sector, d0, phi0, c


CHUNK_EVENTS = 2048


def make_batch(spec, n_events: int, consts: Constants | None = None, seed: int | None = None) -> Batch:
    """Generate ``n_events`` events of ``spec`` (a BatchSpec or a SPECS key).

    Events are produced in fixed chunks of 2048 with per-chunk streams, so the
    result depends only on (spec, n_events, seed).
    """
    if isinstance(spec, str):
        spec = SPECS[spec]
    if consts is None:
        consts = make_constants(spec.n_sectors)
    seed = spec.seed if seed is None else seed
    parts = []
    first_road = 0
    for ci, e0 in enumerate(range(0, n_events, CHUNK_EVENTS)):
        ne = min(CHUNK_EVENTS, n_events - e0)
        rng = np.random.default_rng([seed, ci])
        part = _gen_chunk(spec, consts, rng, ne, e0, first_road)
        first_road += int(part[2].sum())
        parts.append(part)
    if not parts:
        z = np.zeros(0, np.int64)
        return Batch(np.zeros(0, np.uint32), np.zeros(1, np.uint64), z, np.zeros((0, 6), np.int64), z,
                     np.zeros(0), np.zeros(0), np.zeros(0))
    total = sum(len(p[0]) for p in parts)
    words = np.empty(total, np.uint32)
    offs = [np.zeros(1, np.int64)]
    base = 0
    for p in parts:
        words[base:base + len(p[0])] = p[0]
        offs.append(p[1][1:] + base)
        base += len(p[0])
    event_off = np.concatenate(offs).astype(np.uint64)
    cat = lambda i: np.concatenate([p[i] for p in parts])
    return Batch(words, event_off, cat(2), cat(3), cat(4), cat(5), cat(6), cat(7), spec.xft)


def tile_batch(b: Batch, times: int) -> Batch:
    """`times` copies of batch `b` back to back (event and road ids repeat; the
    word format does not require them to be unique).  Full-size batches of
    the uneven workload are built this way from a smaller draw."""
    n_w = len(b.words)
    words = np.tile(b.words, times)
    step = np.arange(times, dtype=np.uint64)[:, None] * np.uint64(n_w)
    off = (b.event_off[None, :-1] + step).ravel()
    event_off = np.concatenate([off, [np.uint64(n_w * times)]]).astype(np.uint64)
    rep = lambda a: np.concatenate([a] * times)
    return Batch(words, event_off, rep(b.n_roads), rep(b.n_hits), rep(b.sector), rep(b.d0),
                 rep(b.phi0), rep(b.c), b.xft)


def make_tracks_batch(consts: Constants, n_roads: int, seed: int, mode="linear",
                      sigma_scale=0.0, roads_per_event=16):
    """Roads holding exactly one hit per layer from one track (no noise).

    With ``mode='linear'`` and ``sigma_scale=0`` the coordinates follow the
    constants' own linear model up to rounding to an integer LSB.
    """
    rng = np.random.default_rng([seed, 0x7A])
    geo = consts.geometry
    S = consts.n_sectors
    d0 = rng.uniform(-D0_MAX_CM, D0_MAX_CM, n_roads)
    # keep the track inside its sector so the sector-relative azimuth is small
    sector = rng.integers(0, S, n_roads)
    phi0 = geo.centre(sector) + rng.uniform(-0.45, 0.45, n_roads) * geo.sector_width
    pt = rng.uniform(PT_MIN, PT_MAX, n_roads)
    charge = np.where(rng.random(n_roads) < 0.5, -1.0, 1.0)
    c = charge * 0.003 * B_TESLA / pt / 2.0
    xt = true_coords(geo, sector, d0, phi0, c, mode)
    xt = xt + rng.normal(0.0, 1.0, xt.shape) * SIGMA_LSB[None, :] * sigma_scale
    coord = np.clip(np.rint(xt), 0, COORD_MAX).astype(np.uint32)
    n_events = (n_roads + roads_per_event - 1) // roads_per_event
    n_r = np.full(n_events, roads_per_event, np.int64)
    if n_roads % roads_per_event:
        n_r[-1] = n_roads % roads_per_event
    words = []
    offs = [0]
    r = 0
    for e in range(n_events):
        ev = [int(event_word(e, n_r[e]))]
        for _ in range(n_r[e]):
            ev.append(int(road_word(sector[r], r)))
            ev.extend(int(hit_word(l, coord[r, l])) for l in range(6))
            r += 1
        words.extend(ev)
        offs.append(len(words))
    return Batch(np.array(words, np.uint32), np.array(offs, np.uint64), n_r,
                 np.ones((n_roads, 6), np.int64), sector.astype(np.int64), d0, phi0, c)


def truth_in_output_units(consts: Constants, batch: Batch):
    """True (d0, dphi0, c) of each road expressed in output LSB: [R, 3]."""
    dphi0 = batch.phi0 - consts.geometry.centre(batch.sector)
    return np.stack([batch.d0, dphi0, batch.c], axis=1) / consts.unit[None, :]


# --- calibration tracks (FP32 relaxation) ------------------------------------
@dataclass
class CalibSet:
    x: np.ndarray              # float32 [N, 6] coordinates in LSB
    sector: np.ndarray         # int32 [N]
    theta: np.ndarray          # float32 [N, 3] true parameters in output LSB
    F0: np.ndarray             # float32 [S, 6, 6] starting constants (all-layer mask)
    q0: np.ndarray             # float32 [S, 6]
    weight: np.ndarray         # float32 [3] 1/Var(theta_k)


def make_calib(n_tracks: int, consts: Constants, seed: int = BASE_SEED + 3,
               sigma_scale: float = 1.0, perturb: float = 0.02) -> CalibSet:
    """Tracks with known parameters for calibrating FP32 constants.

    The starting constants are the integer table's all-layer rows as floats
    (F / 2^oshift, q * 2^(qshift-oshift)) with a relative perturbation.
    """
    rng = np.random.default_rng([seed, 0xCA])
    geo = consts.geometry
    S = consts.n_sectors
    sector = rng.integers(0, S, n_tracks)
    d0 = rng.uniform(-D0_MAX_CM, D0_MAX_CM, n_tracks)
    phi0 = geo.centre(sector) + rng.uniform(-0.5, 0.5, n_tracks) * geo.sector_width
    pt = rng.uniform(PT_MIN, PT_MAX, n_tracks)
    charge = np.where(rng.random(n_tracks) < 0.5, -1.0, 1.0)
    c = charge * 0.003 * B_TESLA / pt / 2.0
    x = true_coords(geo, sector, d0, phi0, c, "linear")
    x = x + rng.normal(0.0, 1.0, x.shape) * SIGMA_LSB[None, :] * sigma_scale
    x = np.clip(x, 0.0, COORD_MAX)
    dphi0 = phi0 - geo.centre(sector)
    theta = np.stack([d0, dphi0, c], axis=1) / consts.unit[None, :]
    F0 = consts.F[:, 63].astype(np.float64) / 2.0 ** consts.oshift
    q0 = consts.q[:, 63].astype(np.float64) * 2.0 ** (consts.qshift - consts.oshift)
    F0 = F0 * (1.0 + perturb * rng.normal(0.0, 1.0, F0.shape))
    q0 = q0 + perturb * np.abs(q0).mean() * rng.normal(0.0, 1.0, q0.shape)
    weight = 1.0 / theta.var(axis=0)
    return CalibSet(x.astype(np.float32), sector.astype(np.int32), theta.astype(np.float32),
                    F0.astype(np.float32), q0.astype(np.float32), weight.astype(np.float32))
