"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only random-number generation: none of the top-k method's
arithmetic. Both the CUDA path's tests and benchmark and the CPU oracle are
fed from it, so it depends on neither.

Every value is a pure function of (seed, stream, element index) through the
SplitMix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): ``h(i) = mix64(base + (i + 1) * GOLDEN)`` with
``base = mix64(seed * GOLDEN + stream)``. The same bytes therefore come out on
any device and for any chunking. Arithmetic is done in torch ``int64`` with
two's-complement wrap-around and masked logical shifts, which equals the
uint64 definition bit for bit (pinned by the tests against Python integers).

Distributions (Sec. 5 of the paper defines UD = U[0, 2^32-1] and
ND = N(1e8, 10); the rest are the workload recipes of this library):
  uniform_u32, normal_f32, uniform_pm1_f32, ascending_u32, descending_u32,
  all_equal_u32, distinct16_u32, zipf_u32 (s = 1.1 over [0, 2^32)),
  nd_u32 (the paper's ND rounded to the nearest integer).
"""

import math

import torch

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1

CHUNK = 1 << 24


def _s64(c):
    """uint64 constant -> the int64 with the same bits."""
    c &= _MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(x, s):
    """Logical right shift of an int64 tensor holding uint64 bits."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def mix64_int(z):
    """SplitMix64 finaliser on a Python int (reference definition)."""
    z &= _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def _mix64(z):
    z = (z ^ _srl(z, 30)) * _s64(_M1)
    z = (z ^ _srl(z, 27)) * _s64(_M2)
    return z ^ _srl(z, 31)


def base_int(seed, stream):
    return mix64_int((seed * GOLDEN + stream) & _MASK64)


def hash_range(seed, stream, start, count, device="cpu"):
    """int64 tensor of h(i) bits for i in [start, start + count)."""
    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = i * _s64(GOLDEN) + _s64(base_int(seed, stream))
    return _mix64(z)


def hash_int(seed, stream, i):
    """h(i) as a Python int (reference definition)."""
    return mix64_int(base_int(seed, stream) + (i + 1) * GOLDEN)


def _u01_53(h):
    """Uniform double in [0, 1) from the top 53 bits."""
    return _srl(h, 11).to(torch.float64) * (2.0 ** -53)


def _low32(x64):
    """Low 32 bits of an int64 tensor, as an int32 tensor with the same bits."""
    v = x64 & 0xFFFFFFFF
    v = torch.where(v >= (1 << 31), v - (1 << 32), v)
    return v.to(torch.int32)


def _fill(n, device, fn):
    """Run fn(start, count) -> int32/float32 tensor over chunks."""
    out = None
    for s in range(0, n, CHUNK):
        c = min(CHUNK, n - s)
        part = fn(s, c)
        if out is None:
            out = torch.empty(n, dtype=part.dtype, device=device)
        out[s:s + c] = part
    if out is None:
        out = torch.empty(0, dtype=torch.int32, device=device)
    return out


# ---- distributions: each returns a 1-D tensor of 32-bit keys ----------------
# u32 keys are returned as torch.int32 tensors holding the unsigned bits
# (torch has no general uint32 arithmetic); callers tell the library the
# dtype is u32.

def uniform_u32(n, seed, device="cpu"):
    """UD (Sec. 5): U[0, 2^32 - 1], the top 32 bits of h(i)."""
    return _fill(n, device, lambda s, c: _low32(_srl(hash_range(seed, 0, s, c, device), 32)))


def normal_f32(n, seed, device="cpu", mean=0.0, std=1.0):
    """N(mean, std) by Box-Muller (cosine branch) from streams 1 and 2."""
    def part(s, c):
        u1 = 1.0 - _u01_53(hash_range(seed, 1, s, c, device))  # (0, 1]
        u2 = _u01_53(hash_range(seed, 2, s, c, device))
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos((2.0 * math.pi) * u2)
        return (mean + std * z).to(torch.float32)
    return _fill(n, device, part)


def uniform_pm1_f32(n, seed, device="cpu"):
    """U[-1, 1) on a 2^-23 grid (exact in float32)."""
    def part(s, c):
        h = hash_range(seed, 3, s, c, device)
        return (_srl(h, 40).to(torch.float64) * (2.0 ** -23) - 1.0).to(torch.float32)
    return _fill(n, device, part)


def ascending_u32(n, seed, device="cpu"):
    """Strictly increasing: v_i = (i << 2) | (h(i) & 3); needs n <= 2^30."""
    if n > (1 << 30):
        raise ValueError("ascending_u32 needs n <= 2^30")
    def part(s, c):
        i = torch.arange(s, s + c, dtype=torch.int64, device=device)
        return _low32((i << 2) | (hash_range(seed, 4, s, c, device) & 3))
    return _fill(n, device, part)


def descending_u32(n, seed, device="cpu"):
    """Strictly decreasing: the bitwise complement of ascending_u32."""
    return torch.bitwise_not(ascending_u32(n, seed, device))


ALL_EQUAL_VALUE = 0x9E3779B9


def all_equal_u32(n, seed=0, device="cpu"):
    """Every key equal to 0x9E3779B9."""
    return torch.full((n,), _s32(ALL_EQUAL_VALUE), dtype=torch.int32, device=device)


def _s32(v):
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v >= (1 << 31) else v


def distinct16_table(seed):
    """16 distinct u32 values drawn from stream 5 (Python ints)."""
    vals, j = [], 0
    while len(vals) < 16:
        v = hash_int(seed, 5, j) >> 32
        if v not in vals:
            vals.append(v)
        j += 1
    return vals


def distinct16_u32(n, seed, device="cpu"):
    """Each element picks one of 16 seeded distinct values uniformly (top 4 bits of h)."""
    table = torch.tensor([_s32(v) for v in distinct16_table(seed)], dtype=torch.int32,
                         device=device)
    return _fill(n, device, lambda s, c: table[_srl(hash_range(seed, 6, s, c, device), 60)])


def nd_u32(n, seed, device="cpu"):
    """The paper's ND (Sec. 5): N(1e8, 10) rounded to the nearest integer."""
    def part(s, c):
        u1 = 1.0 - _u01_53(hash_range(seed, 1, s, c, device))
        u2 = _u01_53(hash_range(seed, 2, s, c, device))
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos((2.0 * math.pi) * u2)
        return _low32(torch.round(1e8 + 10.0 * z).to(torch.int64))
    return _fill(n, device, part)


ZIPF_S = 1.1
ZIPF_N = 1 << 32
ZIPF_ROUNDS = 8


def _zipf_consts(s, N):
    # Rejection-inversion (Hoermann and Derflinger, "Rejection-inversion to
    # generate variates from monotone discrete distributions", ACM TOMACS 1996)
    # for P(k) ~ k^-s on k = 1..N, with the hat integral H(x) = (x^(1-s) - 1)/(1-s).
    def H(x):
        return (x ** (1.0 - s) - 1.0) / (1.0 - s)

    def Hinv(y):
        return (1.0 + y * (1.0 - s)) ** (1.0 / (1.0 - s))

    def h(x):
        return x ** (-s)

    hx1 = H(1.5) - 1.0
    hN = H(N + 0.5)
    sc = 2.0 - Hinv(H(2.5) - h(2.0))
    return hx1, hN, sc


def zipf_u32(n, seed, device="cpu", s=ZIPF_S):
    """Zipf(s) over [0, 2^32): P(v) ~ (v + 1)^-s, by rejection-inversion.

    Each element draws up to ZIPF_ROUNDS proposals (streams 10, 11, ...) and
    keeps the first accepted one; an element with no accepted proposal keeps
    its last proposal (probability below 1e-8 per element at s = 1.1).
    """
    N = float(ZIPF_N)
    hx1, hN, sc = _zipf_consts(s, N)

    def part(st, c):
        res = torch.zeros(c, dtype=torch.float64, device=device)
        done = torch.zeros(c, dtype=torch.bool, device=device)
        for r in range(ZIPF_ROUNDS):
            u = hN + _u01_53(hash_range(seed, 10 + r, st, c, device)) * (hx1 - hN)
            x = torch.pow(1.0 + u * (1.0 - s), 1.0 / (1.0 - s))
            k = torch.clamp(torch.floor(x + 0.5), 1.0, N)
            acc = ((k - x) <= sc) | (u >= (torch.pow(k + 0.5, 1.0 - s) - 1.0) / (1.0 - s)
                                     - torch.pow(k, -s))
            take = (~done) & (acc | (r == ZIPF_ROUNDS - 1))
            res = torch.where(take, k, res)
            done = done | take
        return _low32(res.to(torch.int64) - 1)
    return _fill(n, device, part)


DISTRIBUTIONS = {
    "uniform": uniform_u32,
    "ascending": ascending_u32,
    "descending": descending_u32,
    "all_equal": all_equal_u32,
    "distinct16": distinct16_u32,
    "zipf": zipf_u32,
    "nd": nd_u32,
}

# The five adversarial inputs of the 2^30-key u32 workload.
ADVERSARIAL = ["ascending", "descending", "all_equal", "distinct16", "zipf"]


def batched_rows(rows, seed, device="cpu", lo_exp=10, hi_exp=22, kmax=1024):
    """Ragged batch recipe: row lengths round(2^U[lo, hi]), k_r uniform in
    [1, min(kmax, n_r)] (stream 20 and 21 per row). Returns (lengths, ks) as
    Python lists; the keys of the batch are ``normal_f32(sum(lengths), seed)``
    with the rows laid out back to back."""
    lens, ks = [], []
    for r in range(rows):
        u = (hash_int(seed, 20, r) >> 11) * (2.0 ** -53)
        nr = int(round(2.0 ** (lo_exp + (hi_exp - lo_exp) * u)))
        kr = 1 + (hash_int(seed, 21, r) >> 11) % min(kmax, nr)
        lens.append(nr)
        ks.append(int(kr))
    return lens, ks
