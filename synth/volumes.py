"""Seeded synthetic volumes with the shapes of the paper's field-map experiments.

Recipe (the paper's datasets are not available, so these stand in for them):

* phantom magnitude: a centred ellipsoid with semi-axes (0.4 Nx, 0.35 Ny, 0.4 Nz),
  magnitude 1 inside and 0.05 outside, zero phase (the image x_l = m of Sec. II);
* field map: a sum of random 3-D Gaussians (centres uniform inside the ellipsoid,
  widths 0.1..0.3 of each axis, random signs and amplitudes in [0.5, 1]) rescaled to
  a stated peak in Hz, optionally plus a sharp step a few voxels inside the +x
  boundary;
* coils: N_c complex Gaussians exp(-|r - c_k|^2 / (2 sigma^2)) e^{i phi_k} with centres
  on a ring of radius 0.6 Nx in the mid-z plane, sigma = 0.35 Nx, phi_k uniform; a
  single coil means s = 1;
* echo images by the signal model of Sec. II (Eq. 1): y_clj = e^{i w_j t_l} s_cj x_j,
  plus complex Gaussian noise whose per-component sigma is rms_object|y| / (sqrt(2)
  10^(SNR/20));
* support mask (Sec. IV): voxel centres inside the ellipsoid (where the magnitude is
  at least 0.1 of its maximum) dilated by a Euclidean ball of radius 2 voxels.

Water-fat volumes (make_wf_volume; Sec. II water-fat case, x_l = m_w + m_f sum_p a_p
e^{i 2 pi f_p t_l}): water and fat amplitude maps are smooth nonnegative sums of Gaussians
over the phantom (water 0.05 outside it, fat 0 outside), the fat spectrum is a seeded
6-peak vector (fat_spectrum), echo times 1.2 + k ms, k = 0..5.

Units: echo times in milliseconds, so the field map w is in rad/ms and
f[Hz] = 1000 w / (2 pi).  Arrays are C-ordered [z][y][x] (x fastest); the echo
images are [L][N_c][z][y][x].
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

TE_MS = (0.0, 2.0, 10.0)


def hz_to_rad_per_ms(f_hz):
    return np.asarray(f_hz, dtype=np.float64) * (2.0 * math.pi / 1000.0)


def rad_per_ms_to_hz(w):
    return np.asarray(w, dtype=np.float64) * (1000.0 / (2.0 * math.pi))


@dataclass
class Volume:
    """One synthetic multi-echo acquisition.

    y      complex [L][N_c][nz][ny][nx]  echo images (complex64 unless asked otherwise)
    smap   complex [N_c][nz][ny][nx] or None (None means s = 1, which needs N_c = 1)
    mask   uint8 [nz][ny][nx]            support mask (1 = unknown voxel)
    te     float64 [L]                   echo times (ms)
    omega_true float64 [nz][ny][nx]      true field map (rad/ms)
    beta   regularisation weight of Eq. 5
    """
    y: np.ndarray
    smap: np.ndarray | None
    mask: np.ndarray
    te: np.ndarray
    omega_true: np.ndarray
    beta: float
    name: str = "volume"
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.mask.shape  # (nz, ny, nx)

    @property
    def nx(self):
        return self.mask.shape[2]

    @property
    def ny(self):
        return self.mask.shape[1]

    @property
    def nz(self):
        return self.mask.shape[0]

    @property
    def ncoil(self):
        return self.y.shape[1]

    @property
    def necho(self):
        return self.y.shape[0]

    @property
    def nvox(self):
        return int(self.mask.size)


def _axis(n):
    return np.arange(n, dtype=np.float64) - (n - 1) / 2.0


def ellipsoid_inside(nx, ny, nz):
    """Boolean [nz][ny][nx]: voxel centres inside the phantom ellipsoid."""
    ax, ay, az = 0.4 * nx, 0.35 * ny, 0.4 * nz
    x = (_axis(nx) / ax) ** 2
    y = (_axis(ny) / ay) ** 2
    z = (_axis(nz) / az) ** 2
    return (z[:, None, None] + y[None, :, None] + x[None, None, :]) <= 1.0


def ellipsoid_mask(nx, ny, nz, dilate=2):
    """Support mask: the ellipsoid interior dilated by a Euclidean ball."""
    inside = ellipsoid_inside(nx, ny, nz)
    if dilate <= 0:
        return inside.astype(np.uint8)
    from scipy.ndimage import binary_dilation
    r = int(dilate)
    g = np.arange(-r, r + 1)
    ball = (g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2) <= r * r
    return binary_dilation(inside, structure=ball).astype(np.uint8)


def _field_map_hz(rng, nx, ny, nz, nblobs, fmax_hz, step_hz):
    ax, ay, az = 0.4 * nx, 0.35 * ny, 0.4 * nz
    xs, ys, zs = _axis(nx), _axis(ny), _axis(nz)
    f = np.zeros((nz, ny, nx), dtype=np.float64)
    for _ in range(nblobs):
        while True:  # centre uniform inside the ellipsoid (rejection)
            u = rng.uniform(-1.0, 1.0, size=3)
            if float(u @ u) <= 1.0:
                break
        c = (u[0] * ax, u[1] * ay, u[2] * az)
        sig = rng.uniform(0.1, 0.3, size=3) * np.array([nx, ny, nz], dtype=np.float64)
        amp = rng.uniform(0.5, 1.0) * (1.0 if rng.uniform() < 0.5 else -1.0)
        gx = np.exp(-0.5 * ((xs - c[0]) / sig[0]) ** 2)
        gy = np.exp(-0.5 * ((ys - c[1]) / sig[1]) ** 2)
        gz = np.exp(-0.5 * ((zs - c[2]) / sig[2]) ** 2)
        f += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    peak = float(np.max(np.abs(f)))
    if peak > 0:
        f *= fmax_hz / peak
    if step_hz:
        xb = ax - 3.0  # plane 3 voxels inside the +x boundary of the ellipsoid
        f[:, :, xs > xb] += step_hz
    return f


def _coil_maps(rng, nx, ny, nz, ncoil):
    xs, ys, zs = _axis(nx), _axis(ny), _axis(nz)
    rad = 0.6 * nx
    sig = 0.35 * nx
    phases = rng.uniform(0.0, 2.0 * math.pi, size=ncoil)
    s = np.empty((ncoil, nz, ny, nx), dtype=np.complex128)
    gz = np.exp(-0.5 * (zs / sig) ** 2)  # centres lie in the mid-z plane
    for k in range(ncoil):
        ang = 2.0 * math.pi * k / ncoil
        cx, cy = rad * math.cos(ang), rad * math.sin(ang)
        gx = np.exp(-0.5 * ((xs - cx) / sig) ** 2)
        gy = np.exp(-0.5 * ((ys - cy) / sig) ** 2)
        s[k] = (gz[:, None, None] * gy[None, :, None] * gx[None, None, :]) * np.exp(1j * phases[k])
    return s


def make_volume(nx, ny, nz, ncoil=1, te=TE_MS, snr_db=20.0, seed=0, fmax_hz=150.0,
                nblobs=4, step_hz=0.0, beta=2.0 ** -3, dtype=np.complex64, name=None,
                dilate=2):
    """Draw one seeded volume (see the module docstring for the recipe)."""
    rng = np.random.default_rng(seed)
    te = np.asarray(te, dtype=np.float64)
    L = te.size
    inside = ellipsoid_inside(nx, ny, nz)
    mag = np.where(inside, 1.0, 0.05)
    f_hz = _field_map_hz(rng, nx, ny, nz, nblobs, fmax_hz, step_hz)
    omega = hz_to_rad_per_ms(f_hz)
    smap = _coil_maps(rng, nx, ny, nz, ncoil) if ncoil > 1 else None
    # noise-free images, then the object rms of |y| sets the noise level
    y = np.empty((L, ncoil, nz, ny, nx), dtype=dtype)
    sq = 0.0
    cnt = 0
    for l in range(L):
        ph = np.exp(1j * omega * te[l]) * mag
        for c in range(ncoil):
            yc = ph * smap[c] if smap is not None else ph
            y[l, c] = yc
            sq += float(np.sum(np.abs(yc[inside]) ** 2))
            cnt += int(inside.sum())
    rms = math.sqrt(sq / max(cnt, 1))
    sigma_n = rms / (math.sqrt(2.0) * 10.0 ** (snr_db / 20.0))
    rdt = np.float32 if dtype == np.complex64 else np.float64
    for l in range(L):
        for c in range(ncoil):
            nz_ = rng.standard_normal((2, nz, ny, nx), dtype=rdt)
            y[l, c] += (sigma_n * nz_[0] + 1j * sigma_n * nz_[1]).astype(dtype)
    mask = ellipsoid_mask(nx, ny, nz, dilate=dilate)
    smap_out = smap.astype(dtype) if smap is not None else None
    return Volume(y=y, smap=smap_out, mask=mask, te=te, omega_true=omega, beta=float(beta),
                  name=name or f"{nx}x{ny}x{nz}_c{ncoil}",
                  meta=dict(seed=seed, snr_db=snr_db, fmax_hz=fmax_hz, step_hz=step_hz,
                            nblobs=nblobs, sigma_n=sigma_n))


GYRO_MHZ_PER_T = 42.577478  # proton gyromagnetic ratio / (2 pi)


def fat_spectrum(seed=3003, npeak=6, field_t=3.0):
    """Seeded multipeak fat model for field strength field_t: peak offsets in ppm relative
    to water spanning -3.8 .. +0.6 (both ends fixed, the others uniform in between) and
    relative amplitudes drawn from a Dirichlet distribution whose largest weight sits on the
    peak nearest -3.4 ppm, so they sum to 1.  Returns (amps, freqs) with freqs in cycles per
    ms (kHz) and the ppm offsets for the record."""
    rng = np.random.default_rng(seed)
    inner = np.sort(rng.uniform(-3.8, 0.6, size=npeak - 2))
    ppm = np.concatenate([[-3.8], inner, [0.6]])
    conc = np.ones(npeak)
    conc[int(np.argmin(np.abs(ppm + 3.4)))] = 8.0
    amps = rng.dirichlet(conc)
    freqs_khz = ppm * GYRO_MHZ_PER_T * field_t / 1000.0  # ppm x MHz = Hz
    return amps, freqs_khz, ppm


def _smooth_nonneg(rng, nx, ny, nz, nblobs):
    """Sum of positive 3-D Gaussians centred in the ellipsoid, scaled to a maximum of 1."""
    ax, ay, az = 0.4 * nx, 0.35 * ny, 0.4 * nz
    xs, ys, zs = _axis(nx), _axis(ny), _axis(nz)
    f = np.zeros((nz, ny, nx), dtype=np.float64)
    for _ in range(nblobs):
        while True:
            u = rng.uniform(-1.0, 1.0, size=3)
            if float(u @ u) <= 1.0:
                break
        c = (u[0] * ax, u[1] * ay, u[2] * az)
        sig = rng.uniform(0.15, 0.4, size=3) * np.array([nx, ny, nz], dtype=np.float64)
        amp = rng.uniform(0.3, 1.0)
        gx = np.exp(-0.5 * ((xs - c[0]) / sig[0]) ** 2)
        gy = np.exp(-0.5 * ((ys - c[1]) / sig[1]) ** 2)
        gz = np.exp(-0.5 * ((zs - c[2]) / sig[2]) ** 2)
        f += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return f / max(float(f.max()), 1e-30)


WF_TE_MS = tuple(1.2 + k * 1.0 for k in range(6))


def make_wf_volume(nx, ny, nz, ncoil=1, te=WF_TE_MS, snr_db=20.0, seed=0, fmax_hz=200.0, nblobs=4,
                   beta=2.0 ** -7, fat=None, dtype=np.complex64, name=None, dilate=2, noise=True):
    """Water-fat acquisition by Eq. 1 with x_l = m_w + m_f sum_p a_p e^{i 2 pi f_p t_l}.
    meta holds the true water and fat maps and the fat model (amps, freqs in kHz, ppm)."""
    rng = np.random.default_rng(seed)
    te = np.asarray(te, dtype=np.float64)
    L = te.size
    inside = ellipsoid_inside(nx, ny, nz)
    water = np.where(inside, 0.2 + 0.8 * _smooth_nonneg(rng, nx, ny, nz, nblobs), 0.05)
    fatm = np.where(inside, _smooth_nonneg(rng, nx, ny, nz, nblobs), 0.0)
    amps, freqs, ppm = fat if fat is not None else fat_spectrum()
    f_hz = _field_map_hz(rng, nx, ny, nz, nblobs, fmax_hz, 0.0)
    omega = hz_to_rad_per_ms(f_hz)
    smap = _coil_maps(rng, nx, ny, nz, ncoil) if ncoil > 1 else None
    y = np.empty((L, ncoil, nz, ny, nx), dtype=dtype)
    sq = 0.0
    cnt = 0
    for l in range(L):
        phi_l = complex(np.sum(amps * np.exp(2j * math.pi * freqs * te[l])))
        x = water + fatm * phi_l
        ph = np.exp(1j * omega * te[l]) * x
        for c in range(ncoil):
            yc = ph * smap[c] if smap is not None else ph
            y[l, c] = yc
            sq += float(np.sum(np.abs(yc[inside]) ** 2))
            cnt += int(inside.sum())
    rms = math.sqrt(sq / max(cnt, 1))
    sigma_n = rms / (math.sqrt(2.0) * 10.0 ** (snr_db / 20.0)) if noise else 0.0
    rdt = np.float32 if dtype == np.complex64 else np.float64
    if noise:
        for l in range(L):
            for c in range(ncoil):
                nz_ = rng.standard_normal((2, nz, ny, nx), dtype=rdt)
                y[l, c] += (sigma_n * nz_[0] + 1j * sigma_n * nz_[1]).astype(dtype)
    mask = ellipsoid_mask(nx, ny, nz, dilate=dilate)
    smap_out = smap.astype(dtype) if smap is not None else None
    return Volume(y=y, smap=smap_out, mask=mask, te=te, omega_true=omega, beta=float(beta),
                  name=name or f"wf_{nx}x{ny}x{nz}_c{ncoil}",
                  meta=dict(seed=seed, snr_db=snr_db, fmax_hz=fmax_hz, nblobs=nblobs, sigma_n=sigma_n,
                            water=water, fat=fatm, fat_amps=np.asarray(amps), fat_freqs_khz=np.asarray(freqs),
                            fat_ppm=np.asarray(ppm)))


def wf_config(seed=1003, **kw):
    """192x192x64, 1 coil, 6 echoes 1.2..6.2 ms, +-200 Hz smooth field, SNR 20 dB, water-fat."""
    return make_wf_volume(192, 192, 64, ncoil=1, snr_db=20.0, seed=seed, fmax_hz=200.0, nblobs=4,
                          name="wf_192x192x64_c1", **kw)


def small_config(seed=1001, **kw):
    """64x64x16, single coil, echoes 0/2/10 ms, +-150 Hz from 4 Gaussians, SNR 20 dB."""
    return make_volume(64, 64, 16, ncoil=1, snr_db=20.0, seed=seed, fmax_hz=150.0, nblobs=4,
                       name="small_64x64x16_c1", **kw)


def full_config(seed=1002, **kw):
    """256x256x128, 8 coils, echoes 0/2/10 ms, +-250 Hz mixture + 40 Hz step, SNR 15 dB."""
    return make_volume(256, 256, 128, ncoil=8, snr_db=15.0, seed=seed, fmax_hz=250.0,
                       nblobs=6, step_hz=40.0, name="full_256x256x128_c8", **kw)


def full1_config(seed=1002, **kw):
    """256x256x128, one coil: the full workload's grid and field-map recipe with a single coil
    (the IC sweeps' work does not depend on the coil count; a profiling case that holds
    well under a GB on the device)."""
    return make_volume(256, 256, 128, ncoil=1, snr_db=15.0, seed=seed, fmax_hz=250.0,
                       nblobs=6, step_hz=40.0, name="full_256x256x128_c1", **kw)


def full8_small_config(seed=1007, **kw):
    """64x64x32, 8 coils: the full workload's recipe (echoes 0/2/10 ms, +-250 Hz mixture +
    40 Hz step, SNR 15 dB) at a size whose 100-iteration oracle solve takes minutes."""
    return make_volume(64, 64, 32, ncoil=8, snr_db=15.0, seed=seed, fmax_hz=250.0,
                       nblobs=6, step_hz=40.0, name="full8_64x64x32_c8", **kw)


def diff_config(seed=1005, **kw):
    """128x128x64, 8 coils, echoes 0/2/10 ms (the differentiation workload's shape)."""
    return make_volume(128, 128, 64, ncoil=8, snr_db=20.0, seed=seed, fmax_hz=250.0,
                       nblobs=6, step_hz=40.0, name="diff_128x128x64_c8", **kw)


def phantom_config(seed=1006, **kw):
    """74x74x10, 32 coils, echoes 0/1/2.3 ms, beta 2^-3: the shape of the paper's phantom
    comparison (Sec. IV), with the synthetic phantom and a smooth +-150 Hz field."""
    return make_volume(74, 74, 10, ncoil=32, te=(0.0, 1.0, 2.3), snr_db=20.0, seed=seed, fmax_hz=150.0,
                       nblobs=4, name="phantom_74x74x10_c32", **kw)


def batch_configs(n=32, seed=1004):
    """Sizes/coils/SNRs of n independent volumes from 64x64x16 up to 192x192x96."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(4, 13)) * 16
        ny = int(rng.integers(4, 13)) * 16
        nz = int(rng.integers(1, 7)) * 16
        out.append(dict(nx=nx, ny=ny, nz=nz, ncoil=int(rng.choice([1, 8])),
                        snr_db=float(rng.uniform(10.0, 25.0)), seed=seed * 100 + k))
    return out
