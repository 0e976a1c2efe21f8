"""One integration split in time across ranks (Sec. 2.3.2: consecutive time slices to different
nodes, partial visibilities summed) on CPU: gloo ranks correlate their slices with the FP64
oracle (frames from frame_slice, samples with the delay overlap, fringe phase from the slice's
global first frame) and reduce_visibilities sums them on the host.  The sum equals the oracle on
the whole integration (to FP64 rounding; exactly for the int8 form's integer visibilities), and
a rank that leaves between steps is reported as CORR_E_TIMEOUT on the others within the bound."""
import datetime
import os
import socket
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N_ANT, N_POL, N_FFT = 3, 2, 64


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scales(n_in, n_chan):
    # fixed requantisation scales, the same on every rank
    return np.linspace(0.05, 0.09, n_in * n_chan).reshape(n_in, n_chan)


def _worker(rank, world, port, n_int, leave_after, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle
    from paper_0910_1517_gb300 import timeshard
    from synth import make_config
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=60))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    out = {"rank": rank}
    try:
        s = make_config(2, n_ant=N_ANT, n_pol=N_POL, n_fft=N_FFT, n_int=n_int, seed=4242)   # same on every rank
        tail = s.x.shape[1] - n_int * N_FFT
        t0, nt = timeshard.frame_slice(n_int, world, rank)
        a0, na = timeshard.sample_slice(n_int, N_FFT, world, rank, tail)
        Y = oracle.fengine(s.x[:, a0:a0 + na], N_ANT, N_POL, N_FFT, nt, s.delay, s.phi0, s.rate, g0=t0)
        V = oracle.xengine(Y, N_ANT, N_POL)
        Vi, _ = oracle.xint(oracle.requant(Y, _scales(N_ANT * N_POL, N_FFT // 2)), _scales(N_ANT * N_POL, N_FFT // 2),
                            N_ANT, N_POL)
        dist.barrier()
        out["slice"] = (t0, nt)
        for step in range(2):
            if leave_after is not None and rank == world - 1 and step > leave_after:
                out["left"] = True                     # leaves between steps: nothing in flight
                break
            try:
                out[f"vis{step}"] = timeshard.reduce_visibilities(V, store, step, world, rank, timeout_s=3.0)
                out[f"int{step}"] = timeshard.reduce_visibilities(Vi.astype(np.int32), store, step, world, rank,
                                                                  timeout_s=3.0, prefix="corr-int")
            except timeshard.RankTimeout as e:
                out[f"timeout{step}"] = (e.code, e.missing)
                break
    finally:
        q.put(out)
        # no collective after the steps (a rank may be gone); the store's host, rank 0, stays up
        # until every rank has said it is done with the store
        store.add("done", 1)
        if rank == 0:
            t_end = time.monotonic() + 60
            while store.add("done", 0) < world and time.monotonic() < t_end:
                time.sleep(0.05)
        dist.destroy_process_group()


def _run(world, n_int, leave_after=None):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_int, leave_after, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = {o["rank"]: o for o in (q.get(timeout=240) for _ in range(world))}
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    return res


def _reference(n_int):
    sys.path.insert(0, ROOT)
    import oracle
    from synth import make_config
    s = make_config(2, n_ant=N_ANT, n_pol=N_POL, n_fft=N_FFT, n_int=n_int, seed=4242)
    Y = oracle.fengine(s.x, N_ANT, N_POL, N_FFT, n_int, s.delay, s.phi0, s.rate)
    sc = _scales(N_ANT * N_POL, N_FFT // 2)
    return oracle.xengine(Y, N_ANT, N_POL), oracle.xint(oracle.requant(Y, sc), sc, N_ANT, N_POL)[0]


@pytest.mark.parametrize("world,n_int", [(2, 64), (3, 80)])
def test_split_integration_sums_to_the_whole(world, n_int):
    res = _run(world, n_int)
    V, Vi = _reference(n_int)
    slices = [res[r]["slice"] for r in range(world)]
    assert slices[0][0] == 0 and sum(n for _, n in slices) == n_int
    assert all(slices[r][0] + slices[r][1] == slices[r + 1][0] for r in range(world - 1))
    for r in range(world):
        for step in range(2):
            got = res[r][f"vis{step}"]
            assert np.abs(got - V).max() <= 1e-12 * np.abs(V).max()
            assert np.array_equal(res[r][f"int{step}"], Vi.astype(np.int32))     # exact in int32
            assert np.array_equal(got, res[0][f"vis{step}"])                       # the same bits on every rank


def test_a_rank_that_leaves_is_a_timeout_on_the_others():
    res = _run(3, 48, leave_after=0)
    assert res[2].get("left") and "vis0" in res[2]
    for r in (0, 1):
        assert "vis0" in res[r]                                # step 0 had every rank
        assert res[r]["timeout1"] == (-8, [2])                 # step 1: CORR_E_TIMEOUT naming rank 2


def test_frame_slices():
    from paper_0910_1517_gb300 import timeshard
    for n_int, world in ((8192, 1), (8192, 2), (8192, 3), (8192, 8), (80, 3), (48, 3)):
        sl = [timeshard.frame_slice(n_int, world, r) for r in range(world)]
        assert sum(n for _, n in sl) == n_int and all(n % 16 == 0 and n > 0 for _, n in sl)
        assert all(sl[r][0] + sl[r][1] == sl[r + 1][0] for r in range(world - 1))
        assert max(n for _, n in sl) - min(n for _, n in sl) <= 16
    with pytest.raises(ValueError):
        timeshard.frame_slice(32, 3, 0)                        # fewer 16-frame units than ranks
