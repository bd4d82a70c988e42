"""Seeded synthetic tumour-concentration volumes (input generator only).

The paper's database (50,000 reaction-diffusion simulations at 128^3 in the
SRI24 atlas, Section 3 "Data") and its patients are not available, so every
input here is a seeded surrogate with the same shapes, value range and
compact single-focus structure.  This module holds none of the query's
arithmetic: it only makes volumes, which both the CUDA library and the CPU
oracle then consume byte for byte.

Definition of entry ``e`` of a database with seed ``s`` on an nx x ny x nz grid:

* random numbers: a counter-based SplitMix64 stream (Steele, Lea & Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014).  The
  stream key is ``mix(mix(s + G) ^ (e * H))``; draw ``i`` is
  ``mix(key + (i + 1) * G)`` and a uniform double is its top 53 bits
  times 2^-53.  ``mix`` is the SplitMix64 output function and ``G`` the
  golden-ratio increment.
* brain: the ellipsoid centred at ((nx-1)/2, (ny-1)/2, (nz-1)/2) with
  semi-axes (0.46 nx, 0.40 ny, 0.36 nz).  Its per-row x-range is computed
  once on the host in binary64, so every generator agrees on it exactly.
* parameters theta_e = (cx, cy, cz, R, w, ax, ay, az): the centre is uniform
  in the brain ellipsoid scaled by 0.6 (rejection sampling over fixed draw
  slots 0..191, three draws per attempt; after 64 rejections the brain
  centre is used), R ~ U(5, 25) voxels (draw 192), w ~ U(1, 4) (draw 193),
  per-axis anisotropy a ~ U(0.7, 1.3) (draws 194..196).
* concentration inside the brain, in binary32:
  ``c = 1 / (1 + exp((r - R) / w))`` with ``r = sqrt(sum_i ((x_i - c_i)/a_i)^2)``,
  then ``c = clamp(c + n, 0, 1)`` with voxel noise ``n = u * 0.02 - 0.01`` where
  ``u`` is the top 24 bits of draw ``j`` of the noise stream
  ``mix(key ^ N)`` (``j`` = voxel linear index).  Outside the brain c = +0.
* patients are entries of the same generator with held-out ids
  ``PATIENT_BASE + q`` (q = 1, 2, ...).
* half-precision storage rounds the binary32 value to nearest-even.

Volume layout: [nz][ny][nx], x fastest.

The numpy generator here and the CUDA generator in ``synth.cu`` follow the
same definition; they agree up to the last bits of ``exp`` and are never
compared for parity -- parity always runs both sides on the same bytes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

M64 = (1 << 64) - 1
G = 0x9E3779B97F4A7C15          # SplitMix64 increment
H = 0xD1B54A32D192ED03          # entry-id multiplier for stream keys
N_KEY = 0x6A09E667F3BCC909      # noise sub-stream tweak
DB_SEED = 20220510
PATIENT_BASE = 1 << 40
N_PARAMS = 8
PARAM_NAMES = ("cx", "cy", "cz", "R", "w", "ax", "ay", "az")

_U64 = np.uint64


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    z ^= z >> _U64(30)
    z *= _U64(0xBF58476D1CE4E5B9)
    z ^= z >> _U64(27)
    z *= _U64(0x94D049BB133111EB)
    z ^= z >> _U64(31)
    return z


def _mix_int(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def stream_keys(seed: int, entries) -> np.ndarray:
    """Stream key of each entry id (uint64 array)."""
    e = np.asarray(entries, dtype=np.uint64).reshape(-1)
    base = _U64(_mix_int(seed + G))
    with np.errstate(over="ignore"):
        return _mix_np(base ^ (e * _U64(H)))


def noise_keys(keys: np.ndarray) -> np.ndarray:
    return _mix_np(np.asarray(keys, dtype=np.uint64) ^ _U64(N_KEY))


def _uniform(keys: np.ndarray, draw: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = _mix_np(keys + _U64((draw + 1) * G & M64))
    return (z >> _U64(11)).astype(np.float64) * 2.0 ** -53


def brain_axes(shape):
    nx, ny, nz = shape
    return ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0), (0.46 * nx, 0.40 * ny, 0.36 * nz)


def brain_xrange(shape) -> np.ndarray:
    """Inclusive x-range [xlo, xhi] of the brain ellipsoid per (y, z) row,
    shape [nz*ny, 2] int32; an empty row has xlo > xhi."""
    nx, ny, nz = shape
    (bx, by, bz), (sx, sy, sz) = brain_axes(shape)
    out = np.empty((nz * ny, 2), dtype=np.int32)
    for z in range(nz):
        for y in range(ny):
            q = ((y - by) / sy) ** 2 + ((z - bz) / sz) ** 2
            row = z * ny + y
            if q > 1.0:
                out[row] = (1, 0)
                continue
            h = sx * np.sqrt(1.0 - q)
            lo = int(np.ceil(bx - h))
            hi = int(np.floor(bx + h))
            # make the row exactly the set {x : ((x-bx)/sx)^2 + q <= 1}
            while lo <= hi and ((lo - bx) / sx) ** 2 + q > 1.0:
                lo += 1
            while lo - 1 >= 0 and ((lo - 1 - bx) / sx) ** 2 + q <= 1.0:
                lo -= 1
            while hi >= lo and ((hi - bx) / sx) ** 2 + q > 1.0:
                hi -= 1
            while hi + 1 < nx and ((hi + 1 - bx) / sx) ** 2 + q <= 1.0:
                hi += 1
            out[row] = (max(lo, 0), min(hi, nx - 1))
    return out


_xr_cache: dict = {}


def brain_xrange_cached(shape) -> np.ndarray:
    key = tuple(int(s) for s in shape)
    if key not in _xr_cache:
        _xr_cache[key] = brain_xrange(key)
    return _xr_cache[key]


def entry_params(shape, seed: int, entries) -> np.ndarray:
    """theta for each entry id: float64 [len(entries), 8] =
    (cx, cy, cz, R, w, ax, ay, az)."""
    keys = stream_keys(seed, entries)
    n = keys.shape[0]
    (bx, by, bz), (sx, sy, sz) = brain_axes(shape)
    centre = np.empty((n, 3))
    centre[:] = (bx, by, bz)
    done = np.zeros(n, dtype=bool)
    for attempt in range(64):
        p = np.stack([2.0 * _uniform(keys, 3 * attempt + j) - 1.0 for j in range(3)], axis=1)
        ok = (~done) & ((p * p).sum(axis=1) <= 1.0)
        centre[ok, 0] = bx + 0.6 * sx * p[ok, 0]
        centre[ok, 1] = by + 0.6 * sy * p[ok, 1]
        centre[ok, 2] = bz + 0.6 * sz * p[ok, 2]
        done |= ok
        if done.all():
            break
    theta = np.empty((n, N_PARAMS), dtype=np.float64)
    theta[:, 0:3] = centre
    theta[:, 3] = 5.0 + 20.0 * _uniform(keys, 192)
    theta[:, 4] = 1.0 + 3.0 * _uniform(keys, 193)
    for j in range(3):
        theta[:, 5 + j] = 0.7 + 0.6 * _uniform(keys, 194 + j)
    return theta


def volume_np(shape, theta_row, key: int) -> np.ndarray:
    """One float32 volume [nz, ny, nx] from its parameters and stream key."""
    nx, ny, nz = shape
    xr = brain_xrange_cached(shape)
    f = np.float32
    cx, cy, cz, R, w, ax, ay, az = (f(t) for t in theta_row)
    x = np.arange(nx, dtype=np.float32)[None, None, :]
    y = np.arange(ny, dtype=np.float32)[None, :, None]
    z = np.arange(nz, dtype=np.float32)[:, None, None]
    dx = (x - cx) / ax
    dy = (y - cy) / ay
    dz = (z - cz) / az
    r2 = dx * dx + dy * dy
    r2 = r2 + dz * dz
    r = np.sqrt(r2)
    with np.errstate(over="ignore"):
        c = f(1.0) / (f(1.0) + np.exp((r - R) / w))
    v = nx * ny * nz
    j = np.arange(v, dtype=np.uint64)
    nk = noise_keys(np.array([key], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        h = _mix_np(nk + (j + _U64(1)) * _U64(G))
    u = (h >> _U64(40)).astype(np.float32) * f(2.0 ** -24)
    noise = u * f(0.02) - f(0.01)
    c = c.reshape(-1) + noise
    c = np.minimum(np.maximum(c, f(0.0)), f(1.0))
    xs = np.arange(nx)
    inside = (xs[None, :] >= xr[:, 0:1]) & (xs[None, :] <= xr[:, 1:2])
    c = np.where(inside.reshape(-1), c, f(0.0)).astype(np.float32)
    return c.reshape(nz, ny, nx)


def generate_np(shape, seed: int, entries, dtype=np.float32):
    """Volumes [len(entries), nz, ny, nx] and theta [len(entries), 8] (numpy, CPU).

    ``dtype`` float32, or float16 (rounded to nearest-even)."""
    entries = np.asarray(entries, dtype=np.uint64).reshape(-1)
    theta = entry_params(shape, seed, entries)
    keys = stream_keys(seed, entries)
    nx, ny, nz = shape
    out = np.empty((entries.shape[0], nz, ny, nx), dtype=dtype)
    for i in range(entries.shape[0]):
        out[i] = volume_np(shape, theta[i], int(keys[i])).astype(dtype)
    return out, theta


def database_np(shape, n: int, seed: int = DB_SEED, dtype=np.float32):
    return generate_np(shape, seed, np.arange(n), dtype)


def patients_np(shape, qs, seed: int = DB_SEED, dtype=np.float32):
    qs = np.asarray(qs, dtype=np.uint64).reshape(-1)
    return generate_np(shape, seed, qs + _U64(PATIENT_BASE), dtype)


# ------------------------------------------------- reaction-diffusion inputs
# Inputs of the forward model of Section 2.1 (Eq. 1-2).  The paper simulates
# in the SRI24 atlas (white matter, grey matter, CSF); without it, a
# synthetic atlas stands in: the brain ellipsoid above, white matter inside
# the same ellipsoid scaled by 0.72, grey matter in the rest of the brain,
# and one CSF-filled ventricle ellipsoid at the centre with semi-axes
# (0.08 nx, 0.16 ny, 0.07 nz).  The tissue map holds the relative
# diffusivity m(x): 1 in white matter, 0.1 in grey matter, 0 in CSF and
# outside the brain (the simulation domain is {m > 0}).
TISSUE_WM, TISSUE_GM = 1.0, 0.1
RD_PARAM_NAMES = ("x", "y", "z", "D_w", "rho", "T_end")
N_RD_PARAMS = 6


def brain_tissue(shape) -> np.ndarray:
    """Relative diffusivity m [nz, ny, nx] float32 of the synthetic atlas."""
    nx, ny, nz = shape
    (bx, by, bz), (sx, sy, sz) = brain_axes(shape)
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]

    def inside(ax, ay, az):
        return ((x - bx) / ax) ** 2 + ((y - by) / ay) ** 2 + ((z - bz) / az) ** 2 <= 1.0

    m = np.zeros((nz, ny, nx), dtype=np.float32)
    m[inside(sx, sy, sz)] = np.float32(TISSUE_GM)
    m[inside(0.72 * sx, 0.72 * sy, 0.72 * sz)] = np.float32(TISSUE_WM)
    m[inside(0.08 * nx, 0.16 * ny, 0.07 * nz)] = 0.0
    return m


def rd_params(shape, seed: int, entries) -> np.ndarray:
    """theta = (x, y, z, D_w, rho, T_end) [len(entries), 6] float64 per entry
    id, in voxel and day units.  The seed point is uniform in the brain
    ellipsoid scaled by 0.6 and must round to a voxel of the domain
    (rejection over draw slots 300..491, three per attempt; fallback: the
    white-matter point 0.4 semi-axes right of the centre).  D_w ~ U(0.05, 0.5)
    voxel^2/day (draw 500), rho ~ U(0.025, 0.25) /day (draw 501); the paper
    discards simulations of unrealistic size, so instead of drawing T_end
    freely the front radius R ~ U(6, 30) voxels is drawn (draw 502) and
    T_end is the time at which a Fisher-KPP front from a point source reaches
    it: in three dimensions the front sits near c t - (5 / (2 lambda)) ln t
    with c = 2 sqrt(D_w rho), lambda = sqrt(rho / D_w) (the logarithmic delay
    of a radial front from a point source), solved for t by 30
    fixed-point steps from t = R / c (t >= 1)."""
    keys = stream_keys(seed, entries)
    n = keys.shape[0]
    tissue = brain_tissue(shape)
    (bx, by, bz), (sx, sy, sz) = brain_axes(shape)
    nx, ny, nz = shape
    pos = np.empty((n, 3))
    pos[:] = (bx + 0.4 * sx, by, bz)
    done = np.zeros(n, dtype=bool)
    for attempt in range(64):
        p = np.stack([2.0 * _uniform(keys, 300 + 3 * attempt + j) - 1.0 for j in range(3)],
                     axis=1)
        c = np.stack([bx + 0.6 * sx * p[:, 0], by + 0.6 * sy * p[:, 1], bz + 0.6 * sz * p[:, 2]],
                     axis=1)
        v = np.floor(c + 0.5).astype(np.int64)
        v[:, 0] = np.clip(v[:, 0], 0, nx - 1)
        v[:, 1] = np.clip(v[:, 1], 0, ny - 1)
        v[:, 2] = np.clip(v[:, 2], 0, nz - 1)
        ok = (~done) & ((p * p).sum(axis=1) <= 1.0) & (tissue[v[:, 2], v[:, 1], v[:, 0]] > 0)
        pos[ok] = c[ok]
        done |= ok
        if done.all():
            break
    theta = np.empty((n, N_RD_PARAMS), dtype=np.float64)
    theta[:, 0:3] = pos
    theta[:, 3] = 0.05 + 0.45 * _uniform(keys, 500)
    theta[:, 4] = 0.025 + 0.225 * _uniform(keys, 501)
    radius = 6.0 + 24.0 * _uniform(keys, 502)
    c = 2.0 * np.sqrt(theta[:, 3] * theta[:, 4])
    lam = np.sqrt(theta[:, 4] / theta[:, 3])
    t = radius / c
    for _ in range(30):
        t = (radius + 2.5 / lam * np.log(np.maximum(t, 1.0))) / c
    theta[:, 5] = t
    return theta


# ---------------------------------------------------------------- CUDA generator
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.cu")
_LIB = os.path.join(_HERE, "_build", "libdbqsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA generator for sm_103a into synth/_build/libdbqsynth.so."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["nvcc", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.synth_generate.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_int, P, P]
            lib.synth_generate.restype = ctypes.c_int
            _lib = lib
        return _lib


class DeviceGenerator:
    """Parameters of a range of entries computed once on the host (binary64)
    and uploaded; ``fill`` generates any sub-range of their volumes on the GPU."""

    def __init__(self, shape, seed: int, entries, device="cuda"):
        import torch
        self.shape = tuple(int(s) for s in shape)
        self.entries = np.asarray(entries, dtype=np.uint64).reshape(-1)
        self.theta = entry_params(self.shape, seed, self.entries)
        keys = noise_keys(stream_keys(seed, self.entries))
        self.device = torch.device(device)
        self._theta = torch.from_numpy(self.theta.astype(np.float32)).to(self.device)
        self._keys = torch.from_numpy(keys.view(np.int64)).to(self.device)
        self._xr = torch.from_numpy(brain_xrange_cached(self.shape)).to(self.device)

    def __len__(self):
        return self.entries.shape[0]

    def fill(self, first: int, count: int, out):
        """Write volumes of entries [first, first+count) of this generator into
        ``out`` (contiguous float32 or float16 CUDA tensor) on the current stream."""
        import torch
        nx, ny, nz = self.shape
        if first < 0 or count < 0 or first + count > len(self):
            raise IndexError("entry range outside the generator")
        if not out.is_contiguous() or out.numel() < count * nx * ny * nz:
            raise ValueError("bad output tensor")
        if out.dtype not in (torch.float32, torch.float16):
            raise ValueError("output must be float32 or float16")
        stream = torch.cuda.current_stream(out.device).cuda_stream
        rc = _load().synth_generate(self._theta.data_ptr() + first * 8 * 4,
                                    self._keys.data_ptr() + first * 8, self._xr.data_ptr(),
                                    nx, ny, nz, count, 1 if out.dtype == torch.float16 else 0,
                                    out.data_ptr(), stream)
        if rc != 0:
            raise RuntimeError(f"synth_generate failed: {rc}")
        return out


def generate_device(shape, seed: int, entries, dtype="float32", out=None, device="cuda"):
    """Volumes for ``entries`` generated on the GPU -> (torch tensor
    [n, nz, ny, nx] on ``device``, theta float64 numpy [n, 8]).

    ``out`` may be a preallocated contiguous tensor of the right size."""
    import torch
    gen = DeviceGenerator(shape, seed, entries, device if out is None else out.device)
    nx, ny, nz = gen.shape
    n = len(gen)
    tdt = torch.float16 if dtype in ("float16", np.float16, torch.float16) else torch.float32
    if out is None:
        out = torch.empty((n, nz, ny, nx), dtype=tdt, device=device)
    gen.fill(0, n, out)
    return out, gen.theta
