"""Autotuner of the kernel shapes of a context.

Times candidate shapes of the Chebyshev propagator (electrons per thread x
column groups per CTA) and of the hop kernel (threads per CTA) on a scratch
context with the same model, precision and batch size, from the caller's
state, and sets the fastest on the context.  Results do not depend on the
propagator shape (every output keeps its summation order).  A
mixed-precision context whose default propagator is the tensor-core kernel
keeps it (its arithmetic differs from the SIMT shapes); only the hop kernel
is tuned then.  The hop candidates are the built-in choice (0: in the mixed
path the register-resident Gauss-Jordan kernel where it fits) and LU CTAs
of 256 or 512 threads; the mixed path's two hop algorithms round the FP32
ratios differently (hop probabilities agree to about 1e-7 relative).
Choices are cached per (N, Ne, precision, batch size) in-process.
"""
import numpy as np

from . import iesh as _I

_CACHE = {}


def cheb_candidates(N, Ne, limit=6, precision=0):
    """Propagator shapes ranked by lane and electron-slot efficiency.

    FP64: (ept, G) with ept 1 or 2 electrons per thread and G * N <= 1024
    threads.  Mixed precision: (4, G), 4 orbitals x 4 electrons per thread
    and G * ceil(N / 4) <= 256 threads, two buffers of Np x (8G + 1) floats
    (Np = N rounded up to a multiple of 4) and a ring of 3 x 16 rows of W
    (48 Np floats) in at most 110 KiB; or (32, G), 8 orbitals x 4
    electrons per thread, G * ceil(ceil(N / 4) / 2) <= 256 threads, the same
    buffers in at most 220 KiB."""
    out = []
    if precision == _I.PREC_MIXED:
        nq = -(-N // 4)
        Np = 4 * nq
        # (4, G): one row quad per thread, 110 KiB; (32, G): two, 220 KiB
        for ept, nqh, cap in ((4, nq, 110), (32, -(-nq // 2), 220)):
            for G in range(1, 256 // nqh + 1):
                if G > 1 and (2 * (Np * 8 * G + Np) + 48 * Np) * 4 > cap * 1024:
                    break
                nb = 4 * G
                if nb > 4 * Ne + 3:
                    break
                thr32 = (G * nqh + 31) // 32 * 32
                eff = G * nqh / thr32 * Ne / (-(-Ne // nb) * nb)
                out.append((eff, nb, ept, G))
        out.sort(key=lambda r: (-r[0], -r[1]))
        return [(ept, G) for _, _, ept, G in out[:limit]]
    for ept in (2, 1):
        for G in range(1, 1024 // N + 1):
            nb = G * ept
            if nb > 2 * Ne + 1:
                break
            thr = G * N
            thr32 = (thr + 31) // 32 * 32
            blocks = -(-Ne // nb)
            eff = thr / thr32 * Ne / (blocks * nb)
            out.append((eff, nb, ept, G))
    out.sort(key=lambda r: (-r[0], -r[1]))
    return [(ept, G) for _, _, ept, G in out[:limit]]


def autotune(ctx, x, p, occ, C, dt, steps=3, seed=0):
    """Pick the fastest shapes for `ctx` from the state (x, p, occ, C).

    Returns dict(cheb=(ept, G), hop_threads=..., times={...})."""
    import torch

    key = (ctx.N, ctx.Ne, ctx.precision, int(x.shape[0]), ctx.deflation)
    if key in _CACHE:
        best = _CACHE[key]
        ctx.set_kernel_shape(best["cheb"][0], best["cheb"][1], best["hop_threads"])
        return best
    scratch = _I.Context(ctx.model, int(x.shape[0]), precision=ctx.precision, stream=ctx.stream,
                         deflation=ctx.deflation)
    times_cheb, times_hop = {}, {}

    def trial(ept, G, hop):
        scratch.set_state(x, p, occ, C)
        scratch.set_kernel_shape(ept, G, hop)
        scratch.run(dt, 1, seed)
        scratch.profile(True)
        scratch.run(dt, steps, seed)
        prof = scratch.profile_read()
        scratch.profile(False)
        return prof["propagate"][0], prof["hop"][0]

    default = scratch.kernel_shape()[:2]
    cands = [default] if default[0] in (8, 16) else cheb_candidates(ctx.N, ctx.Ne, precision=ctx.precision)
    for ept, G in cands:
        times_cheb[(ept, G)] = trial(ept, G, 0)[0]
    for hop in (0, 256, 512):
        ept, G = min(times_cheb, key=times_cheb.get)
        times_hop[hop] = trial(ept, G, hop)[1]
    torch.cuda.synchronize()
    scratch.close()
    best = dict(cheb=min(times_cheb, key=times_cheb.get), hop_threads=min(times_hop, key=times_hop.get),
                times=dict(cheb={f"{k}": v for k, v in times_cheb.items()},
                           hop={f"{k}": v for k, v in times_hop.items()}))
    _CACHE[key] = best
    ctx.set_kernel_shape(best["cheb"][0], best["cheb"][1], best["hop_threads"])
    return best
