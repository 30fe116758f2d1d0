"""Uneven batches: trajectories of different bath sizes (one context per
model) and lifetimes (trajectories end on leaving the surface), advanced
together.  Each context keeps a device work list of its live trajectories,
compacted on the device every `compact_every` steps.

Two drivers: the device loop (default) is one launch of a CUDA graph whose
conditional while node repeats a chunk of steps of every context plus the
compactions until no trajectory is live or the step cap is reached (the
library's iesh_ensemble); the host loop captures one chunk with
torch.cuda.graph and replays it, checking the live count on the host
between chunks.  Live trajectory-steps are counted exactly, from the
trajectories' own step counters.
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
        self.ens = None
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

    def live_steps(self):
        """Trajectory-steps taken so far by live trajectories (a trajectory's
        step counter stops when it finishes)."""
        return int(sum(int(c.counters()[0].sum()) for c in self.ctxs))

    def run(self, max_steps, use_graph=True, device_loop=True):
        """Advance until all trajectories finished or max_steps (counted from
        the start, whole chunks); returns the number of live trajectory-steps
        executed by this call.  device_loop: one launch of the library's
        device-side loop; else a host loop replaying a captured chunk
        (use_graph) or running it eagerly."""
        torch = self.torch
        before = self.live_steps()
        if device_loop and use_graph:
            if self.ens is None:
                self.ens = _I.Ensemble(self.ctxs, self.dt, self.chunk, seed=self.seed,
                                       stream=self.stream.cuda_stream)
            todo = max_steps - self.steps_done
            if todo > 0 and self.live() > 0:
                start, _ = self.ens.status()
                self.ens.run(todo)
                done, _ = self.ens.status()  # synchronises the stream
                self.steps_done += done - start
        else:
            with torch.cuda.stream(self.stream):
                while self.steps_done < max_steps:
                    if self.live() == 0:
                        break
                    if use_graph:
                        if self.graph is None:
                            self.capture()
                        self.graph.replay()
                    else:
                        self._eager_chunk()
                    self.steps_done += self.chunk
        torch.cuda.synchronize()
        return self.live_steps() - before

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
        if self.ens is not None:
            self.ens.close()
            self.ens = None
        for c in self.ctxs:
            c.close()
