"""Seeded synthetic inputs for the heat-diffusion workloads.

This module is shared by the oracle side and the GPU side of every test and of
the benchmark. It holds no arithmetic of the method itself (no stencil, no
halo, no time step, no CFL rule): only counter-based random numbers and the
initial/parameter fields that the workloads start from. Both sides receive the
same arrays from here, so their inputs are identical by construction.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter form. The value
number k (0-based) of the stream with key s is mix(s + (k+1)*GAMMA), where mix
is SplitMix64's output finaliser. A field value at global linear index g is
value number g of a stream whose key is itself value number `stream` of the
stream keyed by the seed. A uniform double in [0, 1) is the top 53 bits times
2^-53.

Fields are produced on GLOBAL indices: the caller passes, per axis, the global
index of each local point, so a field scattered over subdomains and the same
field on one undecomposed array hold identical values.

Workload recipes (the physics of Fig. 1 with the randomised variants used by
the test and benchmark configurations):
  * `ci_uniform_c0`: Ci = 1/c0 with c0 uniform in [c0_lo, c0_hi] per point.
  * `ci_uniform`: Ci uniform in [lo, hi] per point.
  * `gaussian_bump`: T0 = base + amp*exp(-|x - 0.5|^2 / (2 sigma^2)), with
    x_d = i_d * l_d/(n_d - 1) from the global index i_d.
  * `sine_modes`: T0 = base + amp * sum_j prod_d sin(pi m_jd x_d) with the
    integer mode numbers m_jd drawn from the seed.
  * `batch_problems`: sizes, conductivities and heat capacities of many
    independent problems.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser on a uint64 array (wraps mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(key: int, k: np.ndarray) -> np.ndarray:
    """Value number k (uint64 array, 0-based) of the SplitMix64 stream whose
    state starts at `key`: mix(key + (k+1)*GAMMA)."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(key & _MASK) + (k + np.uint64(1)) * GAMMA
    return _mix(s)


def stream_key(seed: int, stream: int) -> int:
    """Key of sub-stream `stream` of `seed`: value number `stream` of the
    stream keyed by the seed."""
    return int(splitmix64(seed, np.array([stream], dtype=np.uint64))[0])


def uniform(seed: int, stream: int, g: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) at global linear indices g."""
    v = splitmix64(stream_key(seed, stream), g)
    return (v >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, g: np.ndarray) -> np.ndarray:
    """Standard normal doubles at indices g (Box-Muller on two sub-streams)."""
    u1 = 1.0 - uniform(seed, stream, g)  # (0, 1]
    u2 = uniform(seed, stream + 1, g)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def global_linear_index(gx, gy, gz, n_g) -> np.ndarray:
    """Broadcast per-axis global indices (1-D arrays) into the uint64 global
    linear index gx + n_gx*(gy + n_gy*gz), shaped [z][y][x]."""
    gx = np.asarray(gx, dtype=np.uint64)[None, None, :]
    gy = np.asarray(gy, dtype=np.uint64)[None, :, None]
    gz = np.asarray(gz, dtype=np.uint64)[:, None, None]
    nx, ny = np.uint64(n_g[0]), np.uint64(n_g[1])
    return gx + nx * (gy + ny * gz)


def _coords(gx, gy, gz, n_g, l):
    # an absent dimension (n_g = 1, 2-D and 1-D grids) sits at the centre
    def c(g, n, ll):
        g = np.asarray(g, dtype=np.float64)
        return np.full(g.shape, 0.5 * ll) if n == 1 else g * (ll / (n - 1))
    x, y, z = c(gx, n_g[0], l[0]), c(gy, n_g[1], l[1]), c(gz, n_g[2], l[2])
    return x[None, None, :], y[None, :, None], z[:, None, None]


def ci_uniform_c0(seed, gx, gy, gz, n_g, c0_lo=1.5, c0_hi=2.5, stream=0):
    """Ci = 1/c0, c0 ~ U[c0_lo, c0_hi] per global point; float64 [z][y][x]."""
    u = uniform(seed, stream, global_linear_index(gx, gy, gz, n_g))
    return 1.0 / (c0_lo + (c0_hi - c0_lo) * u)


def ci_uniform(seed, gx, gy, gz, n_g, lo=0.4, hi=0.67, stream=0):
    """Ci ~ U[lo, hi] per global point; float64 [z][y][x]."""
    u = uniform(seed, stream, global_linear_index(gx, gy, gz, n_g))
    return lo + (hi - lo) * u


def gaussian_bump(gx, gy, gz, n_g, l=(1.0, 1.0, 1.0), base=1.7, amp=1.0,
                  sigma=0.1):
    """T0 = base + amp*exp(-((x-.5)^2+(y-.5)^2+(z-.5)^2)/(2 sigma^2))."""
    x, y, z = _coords(gx, gy, gz, n_g, l)
    r2 = (x - 0.5 * l[0]) ** 2 + (y - 0.5 * l[1]) ** 2 + (z - 0.5 * l[2]) ** 2
    return base + amp * np.exp(-r2 / (2.0 * sigma * sigma))


def sine_mode_numbers(seed, count=8, mmax=8, stream=7):
    """Integer mode numbers m in [1, mmax]^3, `count` of them, from the seed."""
    u = uniform(seed, stream, np.arange(3 * count, dtype=np.uint64))
    return (1 + np.floor(u * mmax).astype(np.int64)).reshape(count, 3)


def sine_modes(seed, gx, gy, gz, n_g, l=(1.0, 1.0, 1.0), base=1.7, amp=0.1,
               count=8, mmax=8):
    """T0 = base + amp * sum_j sin(pi mx_j x) sin(pi my_j y) sin(pi mz_j z)."""
    x, y, z = _coords(gx, gy, gz, n_g, l)
    out = np.full(np.broadcast_shapes(x.shape, y.shape, z.shape), base)
    for mx, my, mz in sine_mode_numbers(seed, count, mmax):
        out = out + amp * (np.sin(np.pi * mx * x / l[0]) * np.sin(np.pi * my * y / l[1])
                           * np.sin(np.pi * mz * z / l[2]))
    return out


def ci_smooth(seed, gx, gy, gz, n_g, l=(1.0, 1.0, 1.0), mean=0.53, amp=0.2, modes=4,
              lo=0.4, hi=0.667, stream=13):
    """A smooth random heat-capacity field (the hidden Ci* of the inverse
    problem): mean * (1 + amp * sum_j a_j prod_d sin(pi m_jd x_d)), a_j ~
    U[-1, 1], m_jd in {1, 2, 3}, clipped to [lo, hi]; float64 [z][y][x]."""
    x, y, z = _coords(gx, gy, gz, n_g, l)
    u = uniform(seed, stream, np.arange(4 * modes, dtype=np.uint64)).reshape(modes, 4)
    acc = np.zeros(np.broadcast_shapes(x.shape, y.shape, z.shape))
    for a, mx, my, mz in u:
        m = [1 + int(v * 3) for v in (mx, my, mz)]
        acc = acc + (2 * a - 1) * (np.sin(np.pi * m[0] * x / l[0]) * np.sin(np.pi * m[1] * y / l[1])
                                   * np.sin(np.pi * m[2] * z / l[2]))
    return np.clip(mean * (1 + amp * acc), lo, hi)


def batch_problems(seed, count=256, nmin=32, nmax=192, stream=11):
    """Independent problems of uneven sizes: per problem (nx, ny, nz) with each
    dimension iid uniform on {nmin..nmax}, lam ~ U[0.5, 2] and a constant
    Ci = 1/c0, c0 ~ U[1.5, 2.5]. Returns (sizes int64 [count,3], lam, ci)."""
    k = np.arange(count, dtype=np.uint64)
    span = nmax - nmin + 1
    sizes = np.stack([nmin + np.floor(uniform(seed, stream + d, k) * span).astype(np.int64)
                      for d in range(3)], axis=1)
    lam = 0.5 + 1.5 * uniform(seed, stream + 3, k)
    ci = 1.0 / (1.5 + uniform(seed, stream + 4, k))
    return sizes, lam, ci


def to_f32(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even FP64 -> FP32 (numpy's cast)."""
    return np.ascontiguousarray(x, dtype=np.float64).astype(np.float32)


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """BF16 storage of an FP64 input: FP64 -> FP32 (nearest-even), then
    FP32 -> BF16 (nearest-even on the upper 16 bits). uint16 array."""
    f = to_f32(x).view(np.uint32).astype(np.uint64)
    lsb = (f >> np.uint64(16)) & np.uint64(1)
    r = (f + np.uint64(0x7FFF) + lsb) >> np.uint64(16)
    return r.astype(np.uint16)


def bf16_bits_to_f64(b: np.ndarray) -> np.ndarray:
    """Exact value of BF16 bit patterns as FP64."""
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
