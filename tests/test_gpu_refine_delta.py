"""Incremental refinement (Algorithm 2) through the C ABI against the oracle.

Every step of a refinement chain -- selection, whether the increment was
taken or the refinement fell back to a reconstruction, the guaranteed bound
and the output array -- must equal the oracle's (ipco_refine_delta) bit for
bit: both decode only the new planes with the two lowest loaded digits as
prefix, interpolate the increment from zero in the same operation order and
add it where it is not zero. Small and ragged fields run in process; the
512^3 bench field and the 8 f64 fields of 384x384x256 run against oracle
digests computed by spawned workers."""
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


def new_plane_bytes(of, b_old, b_new):
    """Stream bytes of the planes [b_new, b_old) of every level (oracle)."""
    tot = 0
    for t in range(of.info()["S"]):
        l = of.stage(t)["level"]
        for k in range(b_new[l - 1], b_old[l - 1]):
            tot += of.stream_size(t, k)
    return tot


def run_chain(x, eb, mode, chain, interp=oracle.CUBIC):
    """GPU and oracle side by side; returns the number of incremental steps."""
    of = oracle.compress(x, eb, mode, interp)
    g = ipc.Field.compress(torch.from_numpy(x).cuda(), eb, mode, interp)
    assert g.export() == of.export()
    yo, vo = of.retrieve(*chain[0])
    yg, vg = g.retrieve(*chain[0], refine_mode=ipc.IPC_REFINE_INCREMENTAL)
    torch.cuda.synchronize()
    assert np.array_equal(yg.cpu().numpy().view(np.uint8), yo.view(np.uint8))
    incs = 0
    for kind, v in chain[1:]:
        b_old = vo.selection()[0]
        _, inc = vo.refine_delta(kind, v)
        vg.refine(kind, v)
        torch.cuda.synchronize()
        so, sg = vo.selection(), vg.selection()
        assert sg[0] == so[0], (kind, v)
        assert sg[1] == so[1] and sg[2] == so[2], (kind, v, sg, so)
        if so[0] != b_old:
            ginc, gbytes = vg.refine_info()
            assert ginc == inc
            if inc:
                assert gbytes == new_plane_bytes(of, b_old, so[0])
        incs += inc
        assert np.array_equal(yg.cpu().numpy().view(np.uint8), yo.view(np.uint8)), (kind, v)
        fin = np.isfinite(x)
        err = np.abs(yg.cpu().numpy().astype(np.float64)[fin] - x[fin].astype(np.float64))
        assert err.max() <= sg[2]
    return incs


EB, BR = oracle.EB, oracle.BITRATE


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape", [(70, 45, 530), (33, 700, 61), (3, 5, 1100), (9, 1200),
                                   (2500,)])
def test_eb_chain_matches_oracle(dtype, shape):
    x = synth.random_field(shape, seed=sum(shape), dtype=dtype, kind="smooth")
    eb = 1e-6 if dtype == np.float32 else 1e-10
    chain = [(EB, 1e-1), (EB, 3e-2), (EB, 1e-3), (EB, 1e-4), (EB, 1e-5), (EB, eb)]
    incs = run_chain(x, eb, oracle.REL, chain)
    # f32: these steps change coarse levels, whose increment's rounding margin
    # (strict model) misses every error target, so all of them reconstruct;
    # f64: the margin is small and every step but the last adds an increment
    if dtype == np.float64:
        assert incs >= 4


@pytest.mark.parametrize("interp", [oracle.LINEAR, oracle.CUBIC, oracle.CUBIC_QUAD])
def test_bitrate_chain_with_outliers(interp):
    # non-finite values and two spikes far beyond the quantizer's range are
    # outliers (a finite spike of 1e30 would instead inflate max|x|, and with
    # it every rounding margin, until no selection differs from another)
    x = synth.random_field((40, 36, 300), seed=77, dtype=np.float32, kind="smooth")
    x[3, 5, 7] = np.nan
    x[11, 0, 100] = np.inf
    x[20, 20, 20] = 50.0
    x[8, 16, 64] = -40.0
    of = oracle.compress(x, 1e-6, oracle.ABS, interp)
    m = of.info()["mandatory"] * 8.0 / of.info()["n"]
    chain = [(BR, m + d) for d in (0.25, 0.5, 1.0, 2.0, 4.0, 8.0)]
    assert run_chain(x, 1e-6, oracle.ABS, chain, interp) >= 4


def test_quadratic_boundaries_eb_chain():
    x = synth.random_field((70, 45, 530), seed=31, dtype=np.float64, kind="smooth")
    chain = [(EB, 1e-1), (EB, 3e-2), (EB, 1e-3), (EB, 1e-4), (EB, 1e-5), (EB, 1e-10)]
    assert run_chain(x, 1e-10, oracle.REL, chain, oracle.CUBIC_QUAD) >= 4


def test_auto_mode_follows_element_type():
    """IPC_REFINE_AUTO: an f64 view refines incrementally (as the oracle's
    increment), an f32 view reconstructs (as a fresh retrieval)."""
    for dtype, eb, incremental in ((np.float64, 1e-10, True), (np.float32, 1e-6, False)):
        x = synth.random_field((40, 33, 70), seed=5, dtype=dtype, kind="smooth")
        of = oracle.compress(x, eb, oracle.REL)
        g = ipc.Field.compress(torch.from_numpy(x).cuda(), eb, ipc.IPC_EB_REL)
        yo, vo = of.retrieve(EB, 1e-2)
        yg, vg = g.retrieve(EB, 1e-2, refine_mode=ipc.IPC_REFINE_AUTO)
        for E in (1e-3, 1e-4):
            if incremental:
                vo.refine_delta(EB, E)
            else:
                yo = vo.refine(EB, E)
            vg.refine(EB, E)
            torch.cuda.synchronize()
            assert vg.selection() == vo.selection()
            inc, _ = vg.refine_info()
            assert bool(inc) == incremental
            assert np.array_equal(yg.cpu().numpy().view(np.uint8), yo.view(np.uint8))


def test_mixed_targets_and_fallback():
    # f32, tight eb: the first refinements change coarse levels, whose
    # increment's rounding margin misses the target (reconstruction), the
    # later ones only fine levels (increment)
    x = synth.grf_k53((96, 80, 130), seed=9, dtype=np.float32).numpy()
    chain = [(EB, 1e-1), (BR, 2.0), (EB, 1e-3), (EB, 3e-5), (BR, 12.0), (EB, 1e-6)]
    run_chain(x, 1e-7, oracle.ABS, chain)


@pytest.fixture(scope="module")
def pool():
    n = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as p:
        yield p


def digest(t) -> str:
    return hashlib.sha256(t.cpu().numpy().tobytes()).hexdigest()


def gpu_chain(h, out, chain):
    v = ipc.ipc_retrieve_ex(h, chain[0][0], chain[0][1], out, ipc.IPC_REFINE_INCREMENTAL)
    torch.cuda.synchronize()
    sel, _, bound = ipc.ipc_selection(v)
    steps = [(sel, False, bound, digest(out))]
    for kind, val in chain[1:]:
        ipc.ipc_refine(v, kind, val, out)
        torch.cuda.synchronize()
        sel, _, bound = ipc.ipc_selection(v)
        inc, _ = ipc.ipc_refine_info(v)
        steps.append((sel, inc, bound, digest(out)))
    ipc.ipc_free(v)
    return steps


def test_bench_field_chain_full_size(pool):
    x = synth.grf_k53((512, 512, 512), seed=1002, device="cuda")
    torch.cuda.synchronize()
    chain = [(EB, 1e-1), (EB, 1e-2), (EB, 1e-3), (EB, 1e-4), (EB, 1e-5)]
    res = pool.apply_async(oracle_jobs.compress_delta_chain,
                           ((x.cpu().numpy(), 1e-6, oracle.ABS, chain),))
    g = ipc.Field.compress(x, 1e-6, ipc.IPC_EB_ABS)
    out = torch.empty_like(x)
    got = gpu_chain(g.h, out, chain)
    cont, want = res.get()
    assert hashlib.sha256(g.export()).hexdigest() == cont
    for i, (a, b) in enumerate(zip(got, want)):
        if i > 0:
            assert (a[0], bool(a[1])) == (b[0], bool(b[1])), i
        assert a[2] == b[2] and a[3] == b[3], i
    assert any(bool(s[1]) for s in want[1:])


def test_f64_fields_chain_full_size(pool):
    xs = [synth.sinusoids3d_torch((384, 384, 256), seed=1400 + j) for j in range(8)]
    torch.cuda.synchronize()
    chain = [(EB, 1e-2), (EB, 1e-4), (EB, 1e-6), (EB, 1e-8)]
    want = pool.map(oracle_jobs.compress_delta_chain,
                    [(x.cpu().numpy(), 1e-8, oracle.REL, chain) for x in xs], chunksize=1)
    hs = ipc.ipc_compress_batch(xs, 1e-8, ipc.IPC_EB_REL)
    try:
        out = torch.empty_like(xs[0])
        for i, h in enumerate(hs):
            cont, steps = want[i]
            assert hashlib.sha256(ipc.ipc_export(h)).hexdigest() == cont, i
            got = gpu_chain(h, out, chain)
            for j, (a, b) in enumerate(zip(got, steps)):
                assert a[0] == b[0] and a[2] == b[2] and a[3] == b[3], (i, j)
                if j > 0:
                    assert bool(a[1]) == bool(b[1]), (i, j)
    finally:
        for h in hs:
            ipc.ipc_free(h)
