"""Seeded synthetic inputs shaped like the paper's workloads (host numpy arrays).

This module holds input recipes only -- no arithmetic of the evaluated functions.  Both
the tests (GPU path vs oracle) and bench.py draw their inputs from here.

Recipes (the paper measures on synthetic uniform inputs: Sec. III.A-D):
* ``uniform(lo, hi)``: a real uniform in [lo, hi] (float64 PCG64), rounded to binary32;
* ``loguniform(emin, emax, signed)``: magnitude 2^U(emin, emax), random sign if signed;
* ``domain_bits(func)``: uniform random bit patterns restricted to the function's domain
  of finite, non-trivially-saturated inputs (rejection sampling), plus 1% specials;
* ``expf_mixed``: 90% uniform in [-103.98, 88.73] and 10% from the specials pool;
* ``near_multiples_of_pio2``: binary32 values nearest to k pi/2 and their neighbours;
* ``specials(func)``: zeros, infinities, quiet and signalling NaNs, subnormals, +-FLT_MAX,
  +-FLT_MIN and a few ulps around the function's overflow/underflow boundaries.
Seeds follow seed = 0xC0DE0000 + 256 * config + func_id.
"""
from __future__ import annotations

import numpy as np

FUNCS = [
    "expf", "exp2f", "exp10f", "expm1f", "logf", "log2f", "log10f", "log1pf", "sinf",
    "cosf", "sincosf", "tanf", "asinf", "acosf", "atanf", "sinhf", "coshf", "tanhf",
    "rsqrtf", "exp2", "log", "exp", "log2", "log10", "exp10",
]
F32_FUNCS = FUNCS[:19]
F64_FUNCS = FUNCS[19:]

# Inputs whose results are finite and not trivially saturated (open intervals).
DOMAIN_F32 = {
    "expf": (-103.98, 88.73), "exp2f": (-150.0, 128.0), "exp10f": (-45.16, 38.54),
    "expm1f": (-17.4, 88.73), "logf": (0.0, np.inf), "log2f": (0.0, np.inf),
    "log10f": (0.0, np.inf), "log1pf": (-1.0, np.inf), "sinf": (-np.inf, np.inf),
    "cosf": (-np.inf, np.inf), "sincosf": (-np.inf, np.inf), "tanf": (-np.inf, np.inf),
    "asinf": (-1.0, 1.0), "acosf": (-1.0, 1.0), "atanf": (-np.inf, np.inf),
    "sinhf": (-89.42, 89.42), "coshf": (-89.42, 89.42), "tanhf": (-9.02, 9.02),
    "rsqrtf": (0.0, np.inf),
}
# boundary inputs (bit patterns) around which a few ulps are added to the specials
BOUNDARY_F32 = {
    "expf": [0x42B17217, 0xC2CFF1B4, 0xC2AEAC4F], "exp2f": [0x42FFFFFF, 0xC3160000, 0xC2FC0000],
    "exp10f": [0x421A209A, 0xC2349E35], "expm1f": [0x42B17217, 0xC18AA122],
    "sinhf": [0x42B2D4FC], "coshf": [0x42B2D4FC], "tanhf": [0x41102CB3],
    "log1pf": [0xBF7FFFFF], "asinf": [0x3F7FFFFF], "acosf": [0x3F7FFFFF, 0xBF7FFFFF],
}


def seed_for(config: int, func) -> int:
    fid = FUNCS.index(func) if isinstance(func, str) else int(func)
    return 0xC0DE0000 + 256 * config + fid


def rng_for(config: int, func, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed_for(config, func) + 0x100000000 * salt))


def specials_f32(func: str, rng: np.random.Generator) -> np.ndarray:
    base = [0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0xFFC00001,
            0x7F800001, 0x7FA00000, 0x7F7FFFFF, 0xFF7FFFFF, 0x00800000, 0x80800000,
            0x3F800000, 0xBF800000, 0x00000001, 0x80000001, 0x007FFFFF, 0x807FFFFF]
    sub = rng.integers(1, 0x00800000, 16, dtype=np.uint64).astype(np.uint32)
    sub[8:] |= 0x80000000
    out = [np.array(base, dtype=np.uint32), sub]
    for b in BOUNDARY_F32.get(func, []):
        out.append((np.arange(-4, 5, dtype=np.int64) + b).astype(np.uint32))
        out.append((np.arange(-4, 5, dtype=np.int64) + (b ^ 0x80000000)).astype(np.uint32))
    return np.concatenate(out)


def _in_domain(bits: np.ndarray, func: str) -> np.ndarray:
    lo, hi = DOMAIN_F32[func]
    v = bits.view(np.float32)
    with np.errstate(invalid="ignore"):
        return np.isfinite(v) & (v > lo) & (v < hi)


def domain_bits(func: str, n: int, rng: np.random.Generator, special_frac: float = 0.01) -> np.ndarray:
    """Uniform random bit patterns inside the function's domain, plus specials."""
    ns = int(n * special_frac)
    nd = n - ns
    parts, got = [], 0
    while got < nd:
        b = rng.integers(0, 2**32, int((nd - got) * 2.2) + 1024, dtype=np.uint64).astype(np.uint32)
        b = b[_in_domain(b, func)]
        parts.append(b[: nd - got])
        got += parts[-1].size
    sp = specials_f32(func, rng)
    out = np.concatenate(parts + [np.resize(sp, ns)])
    rng.shuffle(out)
    return out


def uniform(lo: float, hi: float, n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(lo, hi, n).astype(np.float32)


def loguniform(emin: float, emax: float, n: int, rng: np.random.Generator, signed: bool) -> np.ndarray:
    mag = np.exp2(rng.uniform(emin, emax, n))
    if signed:
        mag = np.where(rng.integers(0, 2, n) == 1, -mag, mag)
    with np.errstate(over="ignore"):
        return mag.astype(np.float32)


def expf_mixed(n: int, rng: np.random.Generator) -> np.ndarray:
    """90% uniform in [-103.98, 88.73], 10% drawn round-robin from the specials pool."""
    nu = int(round(n * 0.9))
    u = uniform(-103.98, 88.73, nu, rng).view(np.uint32)
    sp = specials_f32("expf", rng)
    out = np.concatenate([u, np.resize(sp, n - nu)])
    rng.shuffle(out)
    return out.view(np.float32)


def sinf_with_large(n: int, rng: np.random.Generator, frac: float = 0.05) -> np.ndarray:
    """U[-10, 10] with `frac` of the entries replaced by |x| log-uniform in (2^20, 2^127]."""
    x = uniform(-10.0, 10.0, n, rng)
    k = int(n * frac)
    idx = rng.choice(n, k, replace=False)
    x[idx] = loguniform(20.0, 127.0, k, rng, signed=True)
    return x


def near_multiples_of_pio2(n: int, rng: np.random.Generator) -> np.ndarray:
    """Binary32 values nearest to k pi/2 (k log-uniform up to 2^20, random sign) and their neighbours
    within 2 ulps: arguments whose reduced value is tiny, where sin, cos or tan is small or
    huge and the reduction's relative accuracy decides the rounding."""
    k = np.round(np.exp2(rng.uniform(0.0, 20.0, n // 5 + 1)))
    base = (k * (np.pi / 2)).astype(np.float32).view(np.uint32).astype(np.int64)
    out = np.concatenate([base + d for d in (-2, -1, 0, 1, 2)])[:n].astype(np.uint32)
    sign = rng.integers(0, 2, out.size).astype(np.uint32) << np.uint32(31)
    return (out | sign).view(np.float32)


def f64_uniform(lo: float, hi: float, n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(lo, hi, n)


def f64_positive_bits(n: int, rng: np.random.Generator) -> np.ndarray:
    b = rng.integers(1, 0x7FF0000000000000, n, dtype=np.uint64)
    return b.view(np.float64)


# ----------------------------------------------------------------------------- device-side
# For the batching workload (about 3.8e9 inputs) the same recipes run on the GPU with
# torch's seeded generator: uniform random bit patterns restricted to the function's
# domain by rejection.

def domain_bits_device(func: str, n: int, gen, device="cuda"):
    import torch
    lo, hi = DOMAIN_F32[func]
    out = torch.empty(n, dtype=torch.int32, device=device)
    got = 0
    while got < n:
        need = n - got
        cand = torch.randint(-2**31, 2**31, (int(need * 2.2) + 1024,), dtype=torch.int64,
                             device=device, generator=gen).to(torch.int32)
        v = cand.view(torch.float32)
        ok = torch.isfinite(v) & (v > lo) & (v < hi)
        sel = cand[ok][:need]
        out[got:got + sel.numel()] = sel
        got += sel.numel()
    return out.view(torch.float32)


def batch_lengths(count: int, rng: np.random.Generator, lo_log2: float = 6.0, hi_log2: float = 22.0):
    """Lengths log-uniform in [2^lo, 2^hi] and functions uniform over the 19 (config 4)."""
    n = np.round(np.exp2(rng.uniform(lo_log2, hi_log2, count))).astype(np.int64)
    f = rng.integers(0, len(F32_FUNCS), count)
    return n, [F32_FUNCS[i] for i in f]


# ----------------------------------------------------------------------------- bench workloads
# A workload is a list of arrays (label, function, n); bench.py evaluates each array once
# per step.  The inputs are generated on the device (torch's seeded generator) with the
# recipes above; `bench_input_host` draws the same recipe on the host (numpy), for the
# CPU reference timing and for tests.

PRECISION_FUNCS = ("expf", "logf", "sinf", "tanhf", "rsqrtf")
TRIG_FUNCS = ("sinf", "cosf", "sincosf", "tanf")


def bench_arrays(workload: str, scale: int = 0):
    """[(label, func, n)], config dict."""
    if workload == "all19":
        n = (1 << 26) >> scale
        return [(f, f, n) for f in F32_FUNCS], {
            "workload": f"19 binary32 functions x 2^{26 - scale} inputs: domain bit patterns + 1% specials",
            "elems_per_func": n}
    if workload == "precision":
        n = (1 << 28) >> scale
        arrs = []
        for f in PRECISION_FUNCS:
            arrs.append((f + ":u10", f, n))
            arrs.append((f + ":log", f, n))
        arrs.append(("sinf:large", "sinf", n))
        return arrs, {
            "workload": f"expf/logf/sinf/tanhf/rsqrtf x 2^{28 - scale}: (i) U[-10,10], (ii) log-uniform "
                        "[2^-126,2^127] (random sign except logf, rsqrtf); sinf (iii) = (i) with 5% of "
                        "|x| log-uniform in (2^20, 2^127]", "elems_per_array": n}
    if workload == "trig":
        n = (1 << 26) >> scale
        return [(f + ":u10", f, n) for f in TRIG_FUNCS], {
            "workload": f"sinf/cosf/sincosf/tanf x 2^{26 - scale} on U[-10,10] (moderate arguments)",
            "elems_per_array": n}
    if workload == "f64":
        n = (1 << 26) >> scale
        return [("exp2:domain", "exp2", n), ("exp2:u20", "exp2", n), ("log:bits", "log", n),
                ("log:u0.125_8", "log", n), ("exp:edomain", "exp", n), ("log2:bits", "log2", n),
                ("log10:bits", "log10", n), ("exp10:tdomain", "exp10", n)], {
            "workload": f"binary64 x 2^{26 - scale}: exp2 U(-1075,1024) and U[-20,20]; log uniform positive "
                        "finite bit patterns and U[0.125,8]; exp U(-745,710), exp10 U(-324,309), log2 and "
                        "log10 positive finite bit patterns", "elems_per_array": n}
    raise ValueError(f"unknown workload {workload}")


def _set_of(label: str) -> str:
    return label.split(":", 1)[1] if ":" in label else "domain"


def bench_seed(workload: str, label: str, func: str) -> int:
    cfg = {"all19": 2, "precision": 3, "f64": 5, "trig": 6}[workload]
    salt = {"domain": 0, "u10": 0, "log": 1, "large": 2, "u20": 1, "bits": 0, "u0.125_8": 1, "edomain": 0,
            "tdomain": 0}[_set_of(label)]
    return seed_for(cfg, func) + 0x100000000 * salt


def bench_input_host(workload: str, label: str, func: str, n: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(bench_seed(workload, label, func)))
    kind = _set_of(label)
    if workload == "all19":
        return domain_bits(func, n, rng).view(np.float32)
    if workload == "trig":
        return uniform(-10.0, 10.0, n, rng)
    if workload == "precision":
        if kind == "u10":
            return uniform(-10.0, 10.0, n, rng)
        if kind == "log":
            return loguniform(-126.0, 127.0, n, rng, signed=func not in ("logf", "rsqrtf"))
        return sinf_with_large(n, rng, frac=0.05)
    if kind == "domain":
        return f64_uniform(-1075.0, 1024.0, n, rng)
    if kind == "edomain":
        return f64_uniform(-745.0, 710.0, n, rng)
    if kind == "tdomain":
        return f64_uniform(-324.0, 309.0, n, rng)
    if kind == "u20":
        return f64_uniform(-20.0, 20.0, n, rng)
    if kind == "bits":
        return f64_positive_bits(n, rng)
    return f64_uniform(0.125, 8.0, n, rng)


def bench_input_device(workload: str, label: str, func: str, n: int, device="cuda"):
    import torch
    seed = bench_seed(workload, label, func)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    kind = _set_of(label)

    def u(lo, hi, dtype=torch.float64):
        return (torch.rand(n, dtype=torch.float64, device=device, generator=gen) * (hi - lo) + lo).to(dtype)

    def signs(m):
        return torch.randint(0, 2, (m,), device=device, generator=gen).to(torch.bool)

    if workload == "all19":
        x = domain_bits_device(func, n, gen, device=device)
        rng = np.random.Generator(np.random.PCG64(seed + 0x100000000))
        ns = int(n * 0.01)
        sp = np.resize(specials_f32(func, rng), ns)
        pos = torch.from_numpy(rng.choice(n, ns, replace=False)).to(device)
        x[pos] = torch.from_numpy(sp.view(np.float32)).to(device)
        return x
    if workload == "trig":
        return u(-10.0, 10.0, torch.float32)
    if workload == "precision":
        if kind == "log":
            mag = torch.exp2(u(-126.0, 127.0))
            if func not in ("logf", "rsqrtf"):
                mag = torch.where(signs(n), -mag, mag)
            return mag.to(torch.float32)
        x = u(-10.0, 10.0, torch.float32)
        if kind == "large":
            k = int(n * 0.05)
            pos = torch.randperm(n, device=device, generator=gen)[:k]
            mag = torch.exp2(torch.rand(k, dtype=torch.float64, device=device, generator=gen) * 107.0 + 20.0)
            mag = torch.where(signs(k), -mag, mag)
            x[pos] = mag.to(torch.float32)
        return x
    if kind == "domain":
        return u(-1075.0, 1024.0)
    if kind == "edomain":
        return u(-745.0, 710.0)
    if kind == "tdomain":
        return u(-324.0, 309.0)
    if kind == "u20":
        return u(-20.0, 20.0)
    if kind == "bits":
        b = torch.randint(1, 0x7FF0000000000000, (n,), dtype=torch.int64, device=device, generator=gen)
        return b.view(torch.float64)
    return u(0.125, 8.0)
