"""Parity at the full sizes of the other workloads, in the configurations
the bench times: every container and reconstruction is compared, by SHA-256
digest, with the oracle's (run on the host's cores, one field per spawned
worker).
- 64 uneven 2-D f32 fields (16 x 1800x3600, 24 x 900x1800, 24 x 450x900):
  one batched compression at rel eb 1e-4, one batched retrieval at each
  field's eb (log-uniform in [1e-4, 1e-1]);
- 8 f64 fields of 384x384x256, rel eb 1e-8: batched compression, then per
  field a retrieval at 1e-2 refined to 1e-4, 1e-6 and 1e-8;
- a sample of the resident serving fields (k^-5/3, rel eb 1e-6): the three
  smallest and the two largest (the 768^3 class that sets the p99), with eb,
  bitrate and refine requests."""
import hashlib
import multiprocessing as mp
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle  # noqa: E402
from paper_2502_04093_gb300 import ipc, synth  # noqa: E402

import oracle_jobs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_04093_gb300 import build
    build.build()
    oracle.build()


@pytest.fixture(scope="module")
def pool():
    n = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as p:
        yield p


def digest(t) -> str:
    return hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest()


def test_batched_2d_fields_full_size(pool):
    shapes, seeds = synth.zonal_batch(seed=1300)
    xs = [synth.zonal2d_torch(s, sd) for s, sd in zip(shapes, seeds)]
    rng = np.random.default_rng(1303)
    ebs = [float(10 ** rng.uniform(-4, -1)) for _ in xs]
    torch.cuda.synchronize()
    jobs = [(x.cpu().numpy(), 1e-4, oracle.REL, [(oracle.EB, E)]) for x, E in zip(xs, ebs)]
    want = pool.map(oracle_jobs.compress_retrieve, jobs, chunksize=1)
    del jobs
    hs = ipc.ipc_compress_batch(xs, 1e-4, ipc.IPC_EB_REL)
    try:
        outs = [torch.empty_like(x) for x in xs]
        views = ipc.ipc_retrieve_batch(hs, [(ipc.IPC_TARGET_EB, E) for E in ebs], outs,
                                       want_views=True)
        torch.cuda.synchronize()
        for i, (h, v, y) in enumerate(zip(hs, views, outs)):
            cont, [(sel, ydig)] = want[i]
            assert hashlib.sha256(ipc.ipc_export(h)).hexdigest() == cont, i
            assert ipc.ipc_selection(v)[0] == sel, i
            assert digest(y) == ydig, i
            ipc.ipc_free(v)
    finally:
        for h in hs:
            ipc.ipc_free(h)


def test_f64_refine_chain_full_size(pool):
    xs = [synth.sinusoids3d_torch((384, 384, 256), seed=1400 + j) for j in range(8)]
    torch.cuda.synchronize()
    chain = [1e-2, 1e-4, 1e-6, 1e-8]
    want = pool.map(oracle_jobs.compress_refine_chain,
                    [(x.cpu().numpy(), 1e-8, oracle.REL, chain) for x in xs], chunksize=1)
    hs = ipc.ipc_compress_batch(xs, 1e-8, ipc.IPC_EB_REL)
    try:
        out = torch.empty_like(xs[0])
        for i, h in enumerate(hs):
            cont, sels, ydig = want[i]
            assert hashlib.sha256(ipc.ipc_export(h)).hexdigest() == cont, i
            v = ipc.ipc_retrieve(h, ipc.IPC_TARGET_EB, chain[0], out)
            got = [ipc.ipc_selection(v)[0]]
            for E in chain[1:]:
                ipc.ipc_refine(v, ipc.IPC_TARGET_EB, E, out)
                got.append(ipc.ipc_selection(v)[0])
            torch.cuda.synchronize()
            ipc.ipc_free(v)
            assert got == sels, i
            assert digest(out) == ydig, i
    finally:
        for h in hs:
            ipc.ipc_free(h)


@pytest.mark.parametrize("which", ["smallest", "largest"])
def test_serving_fields_sample(pool, which):
    edges = synth.serving_edges(nfields=128, hi=768)
    order = sorted(range(len(edges)), key=lambda j: edges[j])
    pick = order[:3] if which == "smallest" else order[-2:]
    xs = [synth.grf_k53((edges[j],) * 3, seed=1500 + j, device="cuda") for j in pick]
    torch.cuda.synchronize()
    targets = [(oracle.EB, 1e-2), (oracle.BITRATE, 6.5), (oracle.EB, 3e-6)]
    want = pool.map(oracle_jobs.compress_retrieve,
                    [(x.cpu().numpy(), 1e-6, oracle.REL, targets) for x in xs], chunksize=1)
    for x, (cont, res) in zip(xs, want):
        g = ipc.Field.compress(x, 1e-6, ipc.IPC_EB_REL)
        assert hashlib.sha256(g.export()).hexdigest() == cont
        for (kind, v), (sel, ydig) in zip(targets, res):
            y, view = g.retrieve(kind, v)
            torch.cuda.synchronize()
            assert view.selection()[0] == sel
            assert digest(y) == ydig
        # a refine from the first target to the last equals the fresh retrieval
        y, view = g.retrieve(*targets[0])
        view.refine(*targets[2])
        torch.cuda.synchronize()
        assert digest(y) == res[2][1]
