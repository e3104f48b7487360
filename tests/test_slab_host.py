"""x-slab decomposition of one case (Sec. II.B: slabs of whole y-z planes
along x, one per GPU), host side.

* the library's host-only partition, overlap and exchange-size rules;
* the torch.distributed communicator on 3 gloo ranks delivers every exchange
  kind (sum, gather, neighbour halo) exactly as the in-process loopback;
* the phase protocol on real CPU ranks: 2 and 3 processes joined over gloo
  run the package's driver and torch.distributed communicator with each
  slab's phases carried out by the host model of tests/slab_oracle.py (the
  oracle's operators on the slab window, the partition method of the
  pressure equation's x solve, owned flag forces and end fluxes); the
  assembled fields and the flag after the initial projection and 5 steps
  equal the single-domain oracle to 1e-9 (the FP64 parity bound), with bars
  in the first slab and the flag across a cut; with an overlap of 3 planes
  instead of the library's the same run misses the oracle (the check sees
  the overlap width).
"""
import json
import os
import shutil
import socket
import subprocess
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NSTEPS = 5


def workload():
    from paper_2103_08246_gb300 import inputs
    return inputs.small(64, 16, 16, lx=4.0, ly=1.0, lz=1.0, re=100.0, bars_on=True, bar_x=0.5,
                        bar_mesh=0.5, bar_width=0.1, flag_on=True, flag_x_le=1.8, flag_len=1.0,
                        flag_span=0.5, flag_ns=5, flag_nt=5, dt=2e-3)


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2103_08246_gb300 import binding, build
    build.build()
    return binding.load()


def test_split_covers_the_grid_and_windows_stay_inside(lib):
    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300.slab import window
    for nx, R, g in ((64, 2, 11), (64, 3, 11), (100, 4, 12), (512, 8, 15), (40, 1, 0)):
        slabs = [B.ibm_slab_split(nx, R, r, g) for r in range(R)]
        assert slabs[0].x_begin == 0 and slabs[-1].x_end == nx
        for a, b in zip(slabs, slabs[1:]):
            assert a.x_end == b.x_begin
        sizes = [s.x_end - s.x_begin for s in slabs]
        assert max(sizes) - min(sizes) <= 1
        for s in slabs:
            x0, nxw = window(s)
            assert 0 <= x0 and x0 + nxw <= nx
            assert x0 == s.x_begin - (g if s.rank > 0 and R > 1 else 0)
    # a slab shorter than its overlap, too many ranks, bad rank
    for args in ((64, 8, 0, 11), (64, 9, 0, 2), (64, 2, 2, 4), (64, 2, -1, 4)):
        with pytest.raises(B.IBMError):
            B.ibm_slab_split(*args)


def test_overlap_grows_with_the_implicit_decay_length(lib):
    from paper_2103_08246_gb300 import binding as B
    h = 1.0 / 16
    g_small = B.ibm_slab_ghosts(100.0, h, 2e-3)
    g_large = B.ibm_slab_ghosts(100.0, h, 2e-2)
    # r = dt / (2 Re h^2): 0.00256 -> decay factor 2.55e-3, 7 planes to 1e-17, + 4
    assert g_small == 11
    assert g_large > g_small
    rho = np.exp(-2.0 * np.arcsinh(0.5 / np.sqrt(2e-2 / (2 * 100.0 * h * h))))
    assert g_large == int(np.ceil(np.log(1e-17) / np.log(rho))) + 4
    with pytest.raises(B.IBMError):
        B.ibm_slab_ghosts(100.0, h, 0.0)


def test_exchange_sizes(lib):
    from paper_2103_08246_gb300 import binding as B
    grid = B.ibm_grid(64, 16, 32)
    P = 16 * 32
    sl = B.ibm_slab_split(64, 3, 1, 11)
    want = {B.IBM_SLAB_INIT: (B.IBM_XCHG_GATHER, 9 * P, 27 * P),
            B.IBM_SLAB_FORCE: (B.IBM_XCHG_SUM, 3 * 25 + 2, 3 * 25 + 2),
            B.IBM_SLAB_SOLVE: (B.IBM_XCHG_GATHER, 9 * P, 27 * P),
            B.IBM_SLAB_REDUCE: (B.IBM_XCHG_HALO, 2 * P, 2 * P),
            B.IBM_SLAB_PROJECT: (B.IBM_XCHG_HALO, 2 * (4 * 11 + 3) * P, 2 * (4 * 11 + 3) * P),
            B.IBM_SLAB_GHOSTS: (B.IBM_XCHG_NONE, 0, 0)}
    for ph, w in want.items():
        assert B.ibm_slab_plan(grid, 25, sl, ph) == w
    with pytest.raises(B.IBMError):
        B.ibm_slab_plan(grid, 25, sl, 6)


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np
import torch.distributed as dist
from paper_2103_08246_gb300 import binding as B, inputs, slab as S
from slab_oracle import OracleSlab
from test_slab_host import workload, NSTEPS
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world,
                        init_method="tcp://127.0.0.1:" + os.environ["MASTER_PORT"])
wl = workload()
noise = inputs.initial_noise(wl, amp=0.05)
g = B.ibm_slab_ghosts(wl.re, wl.lx / wl.nx, wl.dt)
me = OracleSlab(wl, B.ibm_slab_split(wl.nx, world, rank, g), noise)
comm = S.TorchComm()
S.run_phases([me], comm, S.INIT_SEQUENCE)
for _ in range(NSTEPS):
    S.run_phases([me], comm, S.STEP_SEQUENCE, wl.dt)
u, v, w, p = me.owned()
np.savez(os.path.join({out!r}, "rank%d.npz" % rank), u=u, v=v, w=w, p=p, X=me.X, V=me.V)
dist.barrier()
dist.destroy_process_group()
print(json.dumps({{"rank": rank, "nbars": int(me.Xb.shape[0])}}), flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.fixture(scope="module")
def oracle_run():
    from oracle.solver import OracleSolver
    from paper_2103_08246_gb300 import inputs
    wl = workload()
    ora = OracleSolver(wl, inputs.initial_noise(wl, amp=0.05))
    ora.run(NSTEPS)
    return ora


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_single_domain_oracle(lib, oracle_run, tmp_path, world):
    port = _free_port()
    code = RANK_SCRIPT.format(root=ROOT, out=str(tmp_path))
    env = dict(os.environ, WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
               CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, "-c", code], env=dict(env, RANK=str(r)), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    info = []
    for p in procs:
        out, err = p.communicate(timeout=600)
        assert p.returncode == 0, err[-3000:]
        info.append(json.loads(out.strip().splitlines()[-1]))
    assert info[0]["nbars"] > 0 and info[-1]["nbars"] == 0   # the bars live in the first slab only
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    ora = oracle_run
    for name, ref in zip("uvwp", ora.fields()):
        got = np.concatenate([q[name] for q in parts], axis=0)
        assert got.shape == ref.shape, name
        if name == "p":
            got, ref = got - got.mean(), ref - ref.mean()
        err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1.0)
        assert err < 1e-9, (name, err)
    for q in parts[1:]:   # every rank advanced the same flag
        assert np.array_equal(q["X"], parts[0]["X"]) and np.array_equal(q["V"], parts[0]["V"])
    assert np.abs(parts[0]["X"] - ora.X).max() < 1e-9
    assert np.abs(parts[0]["V"] - ora.V).max() < 1e-9
    # the flag spans a cut between two slabs
    wl = workload()
    cuts = np.cumsum([q["p"].shape[0] for q in parts])[:-1] * wl.lx / wl.nx
    assert any(ora.X[:, 0].min() < c < ora.X[:, 0].max() for c in cuts)


COMM_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch
import torch.distributed as dist
from paper_2103_08246_gb300 import binding as B, slab as S
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world,
                        init_method="tcp://127.0.0.1:" + os.environ["MASTER_PORT"])
comm = S.TorchComm()
def buf(r, n):   # rank r's send buffer: distinct values per rank and element
    return torch.arange(n, dtype=torch.float64) + 1000.0 * (r + 1)
out = {{}}
for kind, n in ((B.IBM_XCHG_SUM, 5), (B.IBM_XCHG_GATHER, 4), (B.IBM_XCHG_HALO, 6)):
    recv_count = n * world if kind == B.IBM_XCHG_GATHER else n
    (got,) = comm.exchange(kind, [buf(rank, n)], recv_count)
    out[kind] = got.tolist()
(none,) = comm.exchange(B.IBM_XCHG_NONE, [None], 0)
out["none"] = none is None
dist.destroy_process_group()
print(json.dumps(out), flush=True)
"""


def test_torch_comm_matches_loopback_on_gloo_ranks():
    """The torch.distributed communicator (3 gloo ranks) delivers every
    exchange kind exactly as the in-process loopback does."""
    import torch

    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300 import slab as S
    world, port = 3, _free_port()
    code = COMM_SCRIPT.format(root=ROOT)
    env = dict(os.environ, WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
               CUDA_VISIBLE_DEVICES="")
    procs = [subprocess.Popen([sys.executable, "-c", code], env=dict(env, RANK=str(r)), cwd=ROOT,
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(world)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    loop = S.LoopbackComm()
    for kind, n in ((B.IBM_XCHG_SUM, 5), (B.IBM_XCHG_GATHER, 4), (B.IBM_XCHG_HALO, 6)):
        sends = [torch.arange(n, dtype=torch.float64) + 1000.0 * (r + 1) for r in range(world)]
        recv_count = n * world if kind == B.IBM_XCHG_GATHER else n
        ref = loop.exchange(kind, sends, recv_count)
        for r in range(world):
            assert outs[r][str(kind)] == ref[r].tolist(), (kind, r)
    assert all(o["none"] for o in outs)
    # halo: the first half comes from the left neighbour's second half, none on rank 0
    assert outs[0][str(B.IBM_XCHG_HALO)][:3] == [0.0, 0.0, 0.0]
    assert outs[1][str(B.IBM_XCHG_HALO)][:3] == [1003.0, 1004.0, 1005.0]


def test_overlap_narrower_than_the_decay_length_is_detected(lib, oracle_run):
    """The same decomposition in one process (loopback exchanges) equals the
    oracle with the library's overlap and misses it with 3 planes: the
    window's wrong ends reach the owned planes through the implicit x factor,
    so the parity check above really tests the overlap width."""
    from paper_2103_08246_gb300 import binding as B
    from paper_2103_08246_gb300 import inputs
    from paper_2103_08246_gb300 import slab as S
    from slab_oracle import OracleSlab
    wl = workload()
    noise = inputs.initial_noise(wl, amp=0.05)

    def run(g):
        ranks = [OracleSlab(wl, B.ibm_slab_split(wl.nx, 2, r, g), noise) for r in range(2)]
        S.run_phases(ranks, S.LoopbackComm(), S.INIT_SEQUENCE)
        for _ in range(NSTEPS):
            S.run_phases(ranks, S.LoopbackComm(), S.STEP_SEQUENCE, wl.dt)
        got = np.concatenate([r.owned()[0] for r in ranks], axis=0)
        ref = oracle_run.fields()[0]
        return np.abs(got - ref).max() / np.abs(ref).max()

    assert run(B.ibm_slab_ghosts(wl.re, wl.lx / wl.nx, wl.dt)) < 1e-12
    assert run(3) > 1e-9
