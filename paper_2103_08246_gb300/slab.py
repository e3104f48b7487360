"""Decomposition of one case into x slabs (Sec. II.B: one-dimensional domain
decomposition over several GPUs), driven through the C ABI's phases.

Each rank holds one slab state (``SlabState``: owned y-z planes plus overlap
planes) and runs the fixed phase sequences of ``include/ibm.h``; between two
phases one buffer moves between the ranks by a plain collective:

  * ``TorchComm``: torch.distributed (NCCL for device buffers, gloo for host
    buffers), one rank per process;
  * ``LoopbackComm``: several ranks in one process (all their states on one
    device), exchanges as device copies; no kernel of one rank waits for
    another, each phase runs to completion on every rank before the exchange.

The arithmetic of every phase runs in the library's kernels; this module
moves buffers and keeps the phase order. ``run_phases`` works with any object
that has ``phase(phase, dt, recv) -> send`` and ``plan(phase)``, so the same
driver and communicators carry the host-side tests of the protocol.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as B
from .inputs import Workload

INIT_SEQUENCE = (B.IBM_SLAB_INIT, B.IBM_SLAB_REDUCE, B.IBM_SLAB_PROJECT, B.IBM_SLAB_GHOSTS)
STEP_SEQUENCE = (B.IBM_SLAB_FORCE, B.IBM_SLAB_SOLVE, B.IBM_SLAB_REDUCE, B.IBM_SLAB_PROJECT,
                 B.IBM_SLAB_GHOSTS)


def window(slab) -> tuple[int, int]:
    """(first global cell plane, planes) of a slab's window."""
    gl = slab.ghosts if slab.rank > 0 else 0
    gr = slab.ghosts if slab.rank < slab.nranks - 1 else 0
    return slab.x_begin - gl, slab.x_end - slab.x_begin + gl + gr


class LoopbackComm:
    """Exchanges among ranks that live in one process (lists of buffers, one
    per rank, in rank order)."""

    def exchange(self, kind, sends, recv_count):
        import torch
        n = len(sends)
        if kind == B.IBM_XCHG_NONE:
            return [None] * n
        if kind == B.IBM_XCHG_SUM:
            total = sends[0].clone()
            for t in sends[1:]:
                total += t
            return [total.clone() for _ in range(n)]
        if kind == B.IBM_XCHG_GATHER:
            cat = torch.cat(sends)
            return [cat.clone() for _ in range(n)]
        if kind == B.IBM_XCHG_HALO:
            out = []
            for r in range(n):
                recv = torch.zeros(recv_count, dtype=sends[r].dtype, device=sends[r].device)
                half = recv_count // 2
                if r > 0:
                    recv[:half] = sends[r - 1][half:]
                if r < n - 1:
                    recv[half:] = sends[r + 1][:half]
                out.append(recv)
            return out
        raise ValueError(f"unknown exchange kind {kind}")


class TorchComm:
    """Exchanges through torch.distributed, one rank per process (the list
    holds this rank's buffer only)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def exchange(self, kind, sends, recv_count):
        import torch
        dist = self.dist
        (send,) = sends
        if kind == B.IBM_XCHG_NONE:
            return [None]
        if kind == B.IBM_XCHG_SUM:
            buf = send.clone()
            dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=self.group)
            return [buf]
        if kind == B.IBM_XCHG_GATHER:
            parts = [torch.empty_like(send) for _ in range(self.size)]
            dist.all_gather(parts, send, group=self.group)
            return [torch.cat(parts)]
        if kind == B.IBM_XCHG_HALO:
            half = recv_count // 2
            recv = torch.zeros(recv_count, dtype=send.dtype, device=send.device)
            ops = []
            if self.rank > 0:
                ops.append(dist.P2POp(dist.isend, send[:half].contiguous(), self.rank - 1, group=self.group))
                ops.append(dist.P2POp(dist.irecv, recv[:half], self.rank - 1, group=self.group))
            if self.rank < self.size - 1:
                ops.append(dist.P2POp(dist.isend, send[half:].contiguous(), self.rank + 1, group=self.group))
                ops.append(dist.P2POp(dist.irecv, recv[half:], self.rank + 1, group=self.group))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
            return [recv]
        raise ValueError(f"unknown exchange kind {kind}")


def run_phases(ranks, comm, sequence, dt=0.0):
    """Run one phase sequence on the local ranks, exchanging between phases."""
    recv = [None] * len(ranks)
    for ph in sequence:
        sends = [r.phase(ph, dt, recv[i]) for i, r in enumerate(ranks)]
        kind, _, recv_count = ranks[0].plan(ph)
        recv = comm.exchange(kind, sends, recv_count)


class SlabState:
    """One slab of a case on the current CUDA device (FP64).

    wl: the global workload; slab: ``binding.ibm_slab`` (e.g. from
    ``binding.ibm_slab_split``); noise: the global initial perturbations
    (u, v, w) or None; this slab's window is cut from them.
    """

    def __init__(self, wl: Workload, slab, noise=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the solver needs a CUDA device")
        B.load()
        self.wl = wl
        self.slab = slab
        self.grid, self.dom, self.bodies = B.structs_from_workload(wl)
        self.x0, self.nxw = window(slab)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self._noise = None
        if noise is not None:
            self._noise = [np.ascontiguousarray(a[self.x0:self.x0 + self.nxw + 1], dtype=np.float64)
                           for a in noise]
        opts = B.ibm_options(B.IBM_FP64, wl.cfl, 2.0, ctypes.c_void_p(self.stream.cuda_stream),
                             *([B._ptr(a) for a in self._noise] if self._noise else [None] * 3))
        self.ws_bytes = B.ibm_slab_workspace_bytes(self.grid, self.dom, self.bodies, opts, slab)
        self.workspace = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        aligned = (self.workspace.data_ptr() + 255) & ~255
        self.state = B.ibm_create_slab(self.grid, self.dom, wl.re, self.bodies, opts, slab,
                                       ctypes.c_void_p(aligned), self.ws_bytes)
        self.nf = wl.flag_ns * wl.flag_nt if wl.flag_on else 0
        self._plans = {ph: B.ibm_slab_plan(self.grid, self.nf, slab, ph) for ph in range(6)}

    def plan(self, phase):
        return self._plans[phase]

    def phase(self, phase, dt, recv):
        import torch
        _, send_count, _ = self._plans[phase]
        send = torch.empty(send_count, dtype=torch.float64, device="cuda") if send_count else None
        rp = ctypes.c_void_p(recv.data_ptr()) if recv is not None else None
        sp = ctypes.c_void_p(send.data_ptr()) if send is not None else None
        # the phase runs on the state's stream; the exchange reads on torch's current stream
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)
        B._check(B.ibm_slab_phase(self.state, phase, dt, rp, sp), "ibm_slab_phase")
        cur.wait_stream(self.stream)
        return send

    def owned_field(self, which):
        """The owned planes of u, v, w (faces x_begin .. x_end - 1, plus the
        outflow face on the last slab) or p (cells x_begin .. x_end - 1)."""
        planes = self.nxw if which == B.IBM_FIELD_P else self.nxw + 1
        out = np.empty((planes, self.wl.ny, self.wl.nz))
        B.ibm_get_field(self.state, which, out)
        lo = self.slab.x_begin - self.x0
        hi = lo + self.slab.x_end - self.slab.x_begin
        if which != B.IBM_FIELD_P and self.slab.rank == self.slab.nranks - 1:
            hi += 1
        return out[lo:hi]

    def flag(self):
        X = np.empty((self.nf, 3))
        V = np.empty((self.nf, 3))
        B.ibm_flag_state(self.state, X, V)
        return X, V

    def close(self):
        if getattr(self, "state", None):
            B.load().ibm_destroy(self.state)
            self.state = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_ranks(wl: Workload, nranks: int, dt: float, noise=None, ghosts=None):
    """All slab states of a case in this process (one device), for the
    loopback communicator."""
    h = wl.lx / wl.nx
    g = B.ibm_slab_ghosts(wl.re, h, dt) if ghosts is None else ghosts
    return [SlabState(wl, B.ibm_slab_split(wl.nx, nranks, r, g), noise) for r in range(nranks)]


def gather_fields(ranks):
    """Global (u, v, w, p) assembled from the slabs' owned planes."""
    out = []
    for which in (B.IBM_FIELD_U, B.IBM_FIELD_V, B.IBM_FIELD_W, B.IBM_FIELD_P):
        out.append(np.concatenate([r.owned_field(which) for r in ranks], axis=0))
    return tuple(out)
