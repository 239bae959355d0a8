"""Seeded synthetic input generators for the median-filter workloads.

This module only draws numbers: it holds none of the median filter's
arithmetic (no window, no sort, no order statistic).  Both sides of every
parity check -- the CPU oracle under ``oracle/`` and the CUDA library in
``paper_1406_1717_gb300/`` -- receive their inputs from here, so they always
see identical bits.  Neither side imports the other.

Generators follow the workloads of the paper's experiments (Section 7.3 lists
asc, desc, r-asc, r-desc, r-large, r-small and r-block) plus the five
configurations this library is measured on:

* ``uniform_f32``      -- i.i.d. float32 uniform [0, 1)
* ``random_walk_f32``  -- Gaussian random walk x_{t+1} = x_t + N(0, 1),
                          accumulated in float64 and cast to float32
* ``uniform_i32``      -- i.i.d. int32 uniform [0, 2^31)
* ``uniform_i64``, ``random_walk_f64`` -- the 64-bit counterparts
* ``batched_signals``  -- many float32 signals with log-uniform lengths and
                          odd window sizes, 10 % impulse noise at +-1e3
* ``distinct_f32``     -- permutation of 0..n-1 scaled by 1e-3 plus N(0, 0.1),
                          redrawn until all values are distinct
* ``serving_requests`` -- Poisson arrivals with log-uniform n and k
* ``request_payload``  -- one served request's samples from SplitMix64

All generators take an explicit integer seed and use numpy's PCG64
``default_rng`` -- except the served payloads, which the request server
draws on the GPU: they follow SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), a counter-based
generator that the device code implements from the same published
definition, so both sides get identical bits.  The default seed is 20140607.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

DEFAULT_SEED = 20140607


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(int(seed))


# ----------------------------------------------------------------------------
# single-signal workloads
# ----------------------------------------------------------------------------
def uniform_f32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """i.i.d. float32 uniform on [0, 1)."""
    return _rng(seed).random(n, dtype=np.float32)


def random_walk_f32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Gaussian random walk x_0 = 0, x_{t+1} = x_t + N(0, 1).

    The cumulative sum is taken in float64 and cast to float32 at the end, so
    the walk does not accumulate float32 rounding drift.  Locally the signal
    is near-sorted: the paper's benign case (Section 7.3, r-asc / r-desc).
    """
    steps = _rng(seed).standard_normal(n)
    steps[0] = 0.0
    return np.cumsum(steps).astype(np.float32)


def uniform_i32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """i.i.d. int32 uniform on [0, 2^31): the paper's r-large generator at 32 bits."""
    return _rng(seed).integers(0, 2 ** 31, size=n, dtype=np.int64).astype(np.int32)


def uniform_i64(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """i.i.d. int64 uniform over the whole int64 range (64-bit r-large)."""
    return _rng(seed).integers(-2 ** 63, 2 ** 63 - 1, size=n, dtype=np.int64, endpoint=True)


def random_walk_f64(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Gaussian random walk x_{t+1} = x_t + N(0, 1) in float64."""
    return np.cumsum(_rng(seed).standard_normal(n))


def distinct_f32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """perm(0..n-1) * 1e-3 + N(0, 0.1) in float32 with all values distinct.

    At n = 65,536 float32 rounding makes a few hundred collisions certain, so
    redrawing the whole signal never succeeds; instead the noise of the
    samples that collide is redrawn until every value is distinct.
    """
    rng = _rng(seed)
    base = rng.permutation(n).astype(np.float64) * 1e-3
    noise = rng.normal(0.0, 0.1, size=n)
    for _ in range(1000):
        x = (base + noise).astype(np.float32)
        order = np.argsort(x, kind="stable")
        dup = np.zeros(n, dtype=bool)
        same = x[order[1:]] == x[order[:-1]]
        dup[order[1:][same]] = True
        if not dup.any():
            return x
        noise[dup] = rng.normal(0.0, 0.1, size=int(dup.sum()))
    raise RuntimeError("could not draw a distinct-valued signal")


# ----------------------------------------------------------------------------
# the seven generators of the paper's Section 7.3
# ----------------------------------------------------------------------------
PAPER_GENERATORS = ("asc", "desc", "r-asc", "r-desc", "r-large", "r-small", "r-block")


def paper_generator(name: str, n: int, seed: int = DEFAULT_SEED,
                    dtype: str = "int32") -> np.ndarray:
    """The input generators listed in the paper's Section 7.3.

    Integer versions follow the stated ranges.  ``r-block`` is under-specified
    in the paper ("piecewise constant data + small uniform random noise"); the
    reading used here: piece lengths uniform in [1, 10^4], piece levels
    uniform over the int32 range shifted to leave room for noise, noise
    uniform in [0, 10^4).  Float versions divide the integer signal by n so the
    values stay exactly representable for n <= 2^24.
    """
    rng = _rng(seed)
    i = np.arange(n, dtype=np.int64)
    if name == "asc":
        v = i
    elif name == "desc":
        v = n - i
    elif name == "r-asc":
        v = i + rng.integers(0, 10 ** 4, size=n)
    elif name == "r-desc":
        v = (n - i) + rng.integers(0, 10 ** 4, size=n)
    elif name == "r-large":
        v = rng.integers(-2 ** 31, 2 ** 31, size=n, dtype=np.int64)
    elif name == "r-small":
        v = rng.integers(0, 10 ** 4, size=n)
    elif name == "r-block":
        v = np.empty(n, dtype=np.int64)
        pos = 0
        while pos < n:
            ln = int(rng.integers(1, 10 ** 4 + 1))
            lvl = int(rng.integers(-2 ** 31, 2 ** 31 - 10 ** 4))
            v[pos:pos + ln] = lvl
            pos += ln
        v += rng.integers(0, 10 ** 4, size=n)
    else:
        raise ValueError(f"unknown generator {name!r}")
    if dtype == "int32":
        return np.clip(v, -2 ** 31, 2 ** 31 - 1).astype(np.int32)
    if dtype == "float32":
        return (v.astype(np.float64) / max(n, 1)).astype(np.float32)
    raise ValueError(dtype)


# ----------------------------------------------------------------------------
# batched and served workloads
# ----------------------------------------------------------------------------
@dataclass
class Batch:
    """Many signals packed end to end in one buffer."""
    x: np.ndarray           # concatenated samples
    n: np.ndarray           # int64 [nseg] signal lengths
    k: np.ndarray           # int32 [nseg] odd window sizes
    x_off: np.ndarray       # int64 [nseg] element offset of each signal in x
    y_off: np.ndarray       # int64 [nseg] element offset of each output in y
    y_total: int            # total outputs, sum(n - k + 1)


def _log_uniform_int(rng, lo: float, hi: float, size=None):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))).astype(np.int64)


def _odd(v):
    v = np.asarray(v, dtype=np.int64)
    return np.where(v % 2 == 0, v + 1, v)


def pack(signals, ks) -> Batch:
    """Pack a list of 1-D arrays (same dtype) and their window sizes."""
    n = np.array([len(s) for s in signals], dtype=np.int64)
    k = np.array(ks, dtype=np.int32)
    x_off = np.zeros(len(signals), dtype=np.int64)
    y_off = np.zeros(len(signals), dtype=np.int64)
    if len(signals) > 1:
        x_off[1:] = np.cumsum(n)[:-1]
        y_off[1:] = np.cumsum(n - k + 1)[:-1]
    x = np.concatenate(signals) if signals else np.zeros(0, np.float32)
    return Batch(x=x, n=n, k=k, x_off=x_off, y_off=y_off,
                 y_total=int((n - k + 1).sum()))


def batched_signals(nseg: int = 4096, seed: int = DEFAULT_SEED,
                    n_lo: int = 1000, n_hi: int = 262144,
                    k_lo: int = 3, k_hi: int = 4095,
                    impulse_frac: float = 0.10, impulse: float = 1e3) -> Batch:
    """float32 signals with log-uniform n in [n_lo, n_hi] and odd log-uniform k.

    k is redrawn while k >= n.  Values are uniform [0, 1) with a fraction
    ``impulse_frac`` of samples replaced by +-impulse (sign 1/2 each), which
    creates many exactly equal values (ties) inside windows.
    """
    rng = _rng(seed)
    sigs, ks = [], []
    for _ in range(nseg):
        n = int(_log_uniform_int(rng, n_lo, n_hi))
        while True:
            k = int(_odd(_log_uniform_int(rng, k_lo, k_hi)))
            if k < n:
                break
        x = rng.random(n, dtype=np.float32)
        hit = rng.random(n) < impulse_frac
        sign = np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
        x[hit] = (impulse * sign[hit]).astype(np.float32)
        sigs.append(x)
        ks.append(k)
    return pack(sigs, ks)


@dataclass
class Request:
    rid: int
    arrival_s: float
    n: int
    k: int
    dtype: str       # "int32" or "float32"
    seed: int        # payload seed: payload(seed) gives the samples


def serving_requests(rate_hz: float = 2000.0, duration_s: float = 60.0,
                     seed: int = DEFAULT_SEED, n_lo: float = 1e3, n_hi: float = 1e7,
                     k_lo: float = 3, k_hi: float = 100001) -> list:
    """Poisson arrivals; n log-uniform [n_lo, n_hi]; odd k log-uniform, k < n."""
    rng = _rng(seed)
    t, rid, out = 0.0, 0, []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        n = int(_log_uniform_int(rng, n_lo, n_hi))
        while True:
            k = int(_odd(_log_uniform_int(rng, k_lo, k_hi)))
            if k < n:
                break
        dt = "int32" if rng.random() < 0.5 else "float32"
        out.append(Request(rid=rid, arrival_s=t, n=n, k=k, dtype=dt,
                           seed=int(rng.integers(0, 2 ** 62))))
        rid += 1
    return out


SPLITMIX_GAMMA = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the SplitMix64 stream started at state
    ``seed``: state_i = seed + i * gamma (mod 2^64), then the published
    finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift 31)."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * SPLITMIX_GAMMA
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def payload_from_bits(z: np.ndarray, dtype: str) -> np.ndarray:
    """int32: the top 16 bits (uniform on [0, 65536)); float32: the top 24
    bits times 2^-24 (uniform on [0, 1), exact in float32)."""
    if dtype == "int32":
        return (z >> np.uint64(48)).astype(np.int32)
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def request_payload(req: Request) -> np.ndarray:
    """Samples of one served request: int32 U[0, 65536) or float32 U[0, 1),
    element i from output i+1 of SplitMix64 seeded with the request's seed."""
    return payload_from_bits(splitmix64(req.seed, req.n), req.dtype)
