"""splitmix64-seeded field values (Steele, Lea & Flood 2014).

A stream with seed s yields z_i = mix(s + (i+1) * 0x9E3779B97F4A7C15) and the
double (z_i >> 11) * 2^-53 in [0, 1).
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed, count, lo=0.0, hi=1.0):
    """count doubles U(lo, hi) from the splitmix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def random_nodal_field(n_nodes, ncomp, seed, lo=-1.0, hi=1.0):
    """i.i.d. U(lo, hi) per degree of freedom, layout [node][comp]."""
    return splitmix64_uniform(seed, n_nodes * ncomp, lo, hi).reshape(n_nodes, ncomp)


def smooth_nodal_field(x, ncomp, seed, modes=4):
    """Low-mode Fourier sum per component, sampled at the points x [N, d].

    f_c(x) = sum_{m in {0..modes-1}^d} a_{c,m} cos(pi m.x + phase_{c,m}),
    a_{c,m} = U(-1,1) / (1 + |m|^2), phase_{c,m} = U(0, 2 pi).
    """
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    grids = np.meshgrid(*([np.arange(modes)] * d), indexing="ij")
    M = np.stack([g_.ravel() for g_ in grids], axis=1).astype(np.float64)   # [nm, d]
    nm = M.shape[0]
    draws = splitmix64_uniform(seed, 2 * ncomp * nm)
    amp = (2.0 * draws[: ncomp * nm] - 1.0).reshape(ncomp, nm) / (1.0 + (M ** 2).sum(1))[None]
    ph = (2.0 * np.pi * draws[ncomp * nm:]).reshape(ncomp, nm)
    # sum_m a cos(pi m.x + ph) = Re sum_m (a e^{i ph}) prod_r e^{i pi m_r x_r}: evaluated as a
    # tensor contraction over the per-axis exponentials (same values up to roundoff)
    coef = (amp * np.exp(1j * ph)).reshape((ncomp,) + (modes,) * d)
    out = np.zeros((x.shape[0], ncomp))
    chunk = 1 << 16
    j = np.arange(modes)
    for s0 in range(0, x.shape[0], chunk):
        xs = x[s0:s0 + chunk]
        E = [np.exp(1j * np.pi * xs[:, r:r + 1] * j[None, :]) for r in range(d)]      # [n, modes]
        if d == 2:
            val = np.einsum("cab,pa,pb->pc", coef, E[0], E[1])
        else:
            val = np.einsum("cabe,pa,pb,pe->pc", coef, E[0], E[1], E[2], optimize=True)
        out[s0:s0 + chunk] = val.real
    return out
