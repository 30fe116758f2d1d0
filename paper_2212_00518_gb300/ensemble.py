"""Uneven batches: trajectories of different bath sizes (one context per
model) and lifetimes (trajectories end on leaving the surface), advanced
together.  Each context keeps a device work list of its live trajectories,
compacted on the device every `compact_every` steps, and the step kernels of
all contexts for a chunk of steps are captured once into one CUDA graph and
replayed until every trajectory has finished or the step cap is reached.
"""
import numpy as np

from . import iesh as _I
from . import tuning as _T


class UnevenBatch:
    def __init__(self, groups, dt, z_done, precision=_I.PREC_MIXED, compact_every=64, seed=0,
                 autotune=False):
        import torch

        self.torch = torch
        self.dt = float(dt)
        self.seed = int(seed)
        self.chunk = int(compact_every)
        self.stream = torch.cuda.Stream()
        self.groups = groups
        self.ctxs = []
        with torch.cuda.stream(self.stream):
            for g in groups:
                md = g["model"]
                n = int(g["x"].shape[0])
                ctx = _I.Context(md, n, precision=precision, z_done=z_done,
                                 compact_every=compact_every, stream=self.stream.cuda_stream)
                occ = np.tile(np.arange(md["Ne"], dtype=np.int16), (n, 1))
                C = np.zeros((n, md["Ne"], md["M"] + 1), dtype=ctx.cdtype)
                C[:, np.arange(md["Ne"]), np.arange(md["Ne"])] = 1.0
                ctx.set_state(np.ascontiguousarray(g["x"]), np.ascontiguousarray(g["p"]), occ, C)
                if autotune:
                    _T.autotune(ctx, g["x"], g["p"], occ, C, self.dt, seed=self.seed)
                    ctx.set_state(np.ascontiguousarray(g["x"]), np.ascontiguousarray(g["p"]),
                                  occ, C)
                self.ctxs.append(ctx)
        self.graph = None
        self.steps_done = 0

    def _eager_chunk(self):
        for ctx in self.ctxs:
            ctx.run(self.dt, self.chunk, self.seed)

    def capture(self):
        """Capture one chunk (compact_every steps of every context, ending with
        the work-list compactions) into a CUDA graph."""
        torch = self.torch
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream):
            self._eager_chunk()
        self.graph = g
        return g

    def live(self):
        return sum(c.live_count() for c in self.ctxs)

    def run(self, max_steps, use_graph=True):
        """Advance until all trajectories finished or max_steps; returns the
        number of live trajectory-steps executed."""
        torch = self.torch
        live_steps = 0
        with torch.cuda.stream(self.stream):
            while self.steps_done < max_steps:
                n_live = self.live()
                if n_live == 0:
                    break
                if use_graph:
                    if self.graph is None:
                        self.capture()
                    self.graph.replay()
                else:
                    self._eager_chunk()
                live_steps += n_live * self.chunk
                self.steps_done += self.chunk
        torch.cuda.synchronize()
        return live_steps

    def results(self):
        """Per trajectory (in the batch's original order): x, p, occ-free
        summary (hops, steps, status)."""
        n = sum(int(g["x"].shape[0]) for g in self.groups)
        x = np.zeros(n)
        p = np.zeros(n)
        hops = np.zeros(n, np.int32)
        nstep = np.zeros(n, np.int64)
        status = np.zeros(n, np.uint32)
        for g, c in zip(self.groups, self.ctxs):
            st = c.get_state()
            ns, hp, _ = c.counters()
            x[g["idx"]] = st["x"]
            p[g["idx"]] = st["p"]
            status[g["idx"]] = st["status"]
            hops[g["idx"]] = hp
            nstep[g["idx"]] = ns
        return dict(x=x, p=p, hops=hops, nstep=nstep, status=status)

    def close(self):
        for c in self.ctxs:
            c.close()
