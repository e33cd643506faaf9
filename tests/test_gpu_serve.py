"""Serving loop: continuous batching must not change any result. Every
served reconstruction equals the same request served alone (bitwise);
admission respects the memory budget; failures come back as statuses."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(240)]

from paper_2502_04093_gb300 import ipc, synth  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_04093_gb300 import build
    build.build()


def drain(server, want, timeout_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < want and time.time() - t0 < timeout_s:
        for c in ipc.ipc_server_poll(server, 64, 20000):
            got[c["ticket"]] = c
    assert len(got) == want, "server did not complete every request"
    return got


@pytest.fixture(scope="module")
def fields():
    shapes = [(40, 48, 36), (64, 64, 64), (33, 70, 21), (96, 80), (128, 129)]
    xs = [torch.from_numpy(synth.random_field(s, seed=i)).cuda() for i, s in enumerate(shapes)]
    fs = [ipc.Field.compress(x, 1e-5, ipc.IPC_EB_REL) for x in xs]
    return xs, fs


@pytest.mark.parametrize("plain,maxv", [(False, 0), (True, 0), (False, 150000)])
def test_results_same_alone_and_in_the_mix(fields, plain, maxv):
    """maxv: batch size limit in values (150000 splits the mix into batches
    of one to a few fields; the 128x129 field fits alone)."""
    xs, fs = fields
    srv = ipc.ipc_server_create(8 << 30, max_inflight=3, nstreams=3, plain=plain,
                                max_batch=1 if plain else 0, max_batch_values=maxv)
    try:
        rng = np.random.default_rng(3)
        reqs = []
        for i in range(40):
            f = int(rng.integers(len(fs)))
            if i % 4 == 3:
                tgt = (ipc.IPC_TARGET_BITRATE, float(rng.uniform(1, 12)))
            else:
                tgt = (ipc.IPC_TARGET_EB, float(10 ** rng.uniform(-5, -1)))
            t = ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, fs[f].h, target=tgt, user_tag=i)
            reqs.append((t, f, tgt))
        got = drain(srv, len(reqs))
        views = {}
        nok = 0
        for t, f, tgt in reqs:
            c = got[t]
            try:
                alone, v = fs[f].retrieve(*tgt)
            except ipc.IpcError as e:  # e.g. a bitrate below the mandatory bytes
                assert c["status"] == e.rc
                continue
            assert c["status"] == 0
            served = ipc.device_view(c["d_out"], xs[f].shape, xs[f].dtype).clone()
            torch.cuda.synchronize()
            assert torch.equal(served, alone)
            assert (c["bytes"], c["bound"]) == v.selection()[1:]
            views[c["view_id"]] = (f, tgt)
            nok += 1
        assert nok >= 30
        # refine chains on live views, submitted all at once (each view's
        # refines must run in order), then compared with fresh retrieval
        vids = list(views)[:8]
        reqs2 = []
        for vid in vids:
            f, tgt = views[vid]
            for E in (1e-3, 1e-4, 1e-5):
                t = ipc.ipc_server_submit(srv, ipc.IPC_REQ_REFINE, view_id=vid,
                                          target=(ipc.IPC_TARGET_EB, E))
                reqs2.append((t, vid, f, E))
        got2 = drain(srv, len(reqs2))
        for vid in vids:
            f, _ = views[vid]
            last = [r for r in reqs2 if r[1] == vid][-1]
            c = got2[last[0]]
            assert c["status"] == 0
            served = ipc.device_view(c["d_out"], xs[f].shape, xs[f].dtype).clone()
            full, _ = fs[f].retrieve(ipc.IPC_TARGET_EB, 1e-5)
            torch.cuda.synchronize()
            assert torch.equal(served, full)
        rel = [ipc.ipc_server_submit(srv, ipc.IPC_REQ_RELEASE, view_id=v) for v in views]
        got3 = drain(srv, len(rel))
        assert all(c["status"] == 0 for c in got3.values())
        assert ipc.ipc_server_stats(srv)["mem_used"] == 0
    finally:
        ipc.ipc_server_destroy(srv)


def test_memory_admission_and_failures(fields):
    xs, fs = fields
    big = fs[1]  # 64^3 f32 = 1 MiB output
    srv = ipc.ipc_server_create(int(1.5 * (1 << 20)), max_inflight=2, nstreams=2)
    try:
        # a request that can never fit the budget fails with ENOMEM
        tiny = ipc.ipc_server_create(1024, max_inflight=1, nstreams=1)
        try:
            t = ipc.ipc_server_submit(tiny, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-2))
            c = drain(tiny, 1)[t]
            assert c["status"] == ipc.IPC_ENOMEM
        finally:
            ipc.ipc_server_destroy(tiny)
        # two 1 MiB views do not fit a 1.5 MiB budget: the second waits for
        # the first one's release
        t1 = ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-2))
        t2 = ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-3))
        c1 = drain(srv, 1)[t1]
        assert c1["status"] == 0
        assert ipc.ipc_server_poll(srv, 8, 50000) == []  # t2 is held back
        ipc.ipc_server_submit(srv, ipc.IPC_REQ_RELEASE, view_id=c1["view_id"])
        got = drain(srv, 2)
        c2 = got[t2]
        assert c2["status"] == 0
        alone, _ = big.retrieve(0, 1e-3)
        torch.cuda.synchronize()
        assert torch.equal(ipc.device_view(c2["d_out"], xs[1].shape, xs[1].dtype), alone)
        # unknown view / bad target statuses
        t = ipc.ipc_server_submit(srv, ipc.IPC_REQ_REFINE, view_id=12345, target=(0, 1e-3))
        assert drain(srv, 1)[t]["status"] == ipc.IPC_EINVAL
        t = ipc.ipc_server_submit(srv, ipc.IPC_REQ_REFINE, view_id=c2["view_id"],
                                  target=(0, 1e-9))
        assert drain(srv, 1)[t]["status"] == ipc.IPC_EBOUND
    finally:
        ipc.ipc_server_destroy(srv)


def test_incremental_refines_same_alone_and_in_the_mix():
    """A server whose refines take the incremental form (Algorithm 2): each
    served refine chain ends bitwise equal to the same chain on a view of
    its own (a canonical retrieval switched to the incremental form, so the
    first refine reconstructs and records the state, the later ones add
    increments), and the selection and bound agree."""
    shapes = [(40, 48, 36), (33, 70, 21), (96, 80)]
    xs = [torch.from_numpy(synth.random_field(s, seed=20 + i, dtype=dt)).cuda()
          for i, s in enumerate(shapes) for dt in (np.float32, np.float64)]
    fs = [ipc.Field.compress(x, 1e-9 if x.dtype == torch.float64 else 1e-6, ipc.IPC_EB_REL)
          for x in xs]
    srv = ipc.ipc_server_create(8 << 30, max_inflight=3, nstreams=3,
                                refine_mode=ipc.IPC_REFINE_INCREMENTAL)
    try:
        ts = [ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, f.h, target=(0, 1e-1))
              for f in fs]
        got = drain(srv, len(ts))
        vids = [got[t]["view_id"] for t in ts]
        assert all(got[t]["status"] == 0 for t in ts)
        chain = [(ipc.IPC_TARGET_EB, 1e-2), (ipc.IPC_TARGET_BITRATE, 6.0),
                 (ipc.IPC_TARGET_EB, 1e-4), (ipc.IPC_TARGET_EB, 1e-5)]
        reqs = [(ipc.ipc_server_submit(srv, ipc.IPC_REQ_REFINE, view_id=vid, target=tg), i, j)
                for j, tg in enumerate(chain) for i, vid in enumerate(vids)]
        got2 = drain(srv, len(reqs))
        for i, f in enumerate(fs):
            out = torch.empty_like(xs[i])
            v = ipc.ipc_retrieve(f.h, 0, 1e-1, out)
            ipc.ipc_view_set_refine_mode(v, ipc.IPC_REFINE_INCREMENTAL)
            for tg in chain:
                ipc.ipc_refine(v, tg[0], tg[1], out)
            torch.cuda.synchronize()
            last = [r for r in reqs if r[1] == i][-1]
            c = got2[last[0]]
            assert c["status"] == 0
            served = ipc.device_view(c["d_out"], xs[i].shape, xs[i].dtype).clone()
            assert torch.equal(served, out), i
            assert (c["bytes"], c["bound"]) == tuple(ipc.ipc_selection(v)[1:]), i
            ipc.ipc_free(v)
        rel = [ipc.ipc_server_submit(srv, ipc.IPC_REQ_RELEASE, view_id=v) for v in vids]
        assert all(c["status"] == 0 for c in drain(srv, len(rel)).values())
    finally:
        ipc.ipc_server_destroy(srv)


def test_stop_completes_what_cannot_run_with_ebusy(fields):
    xs, fs = fields
    big = fs[1]  # 64^3 f32 = 1 MiB output
    srv = ipc.ipc_server_create(int(1.5 * (1 << 20)), max_inflight=2, nstreams=2)
    try:
        t1 = ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-2))
        t2 = ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-3))
        assert drain(srv, 1)[t1]["status"] == 0
        ipc.ipc_server_stop(srv)  # t2 waits for memory that is never released
        assert drain(srv, 1)[t2]["status"] == ipc.IPC_EBUSY
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_server_submit(srv, ipc.IPC_REQ_RETRIEVE, big.h, target=(0, 1e-2))
        assert e.value.rc == ipc.IPC_EBUSY
    finally:
        ipc.ipc_server_destroy(srv)
