"""Serving loop: continuously batched requests give the same results as each request
computed alone, admission respects the HBM budget, and waits time out cleanly."""
import threading

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def make_requests(w, ids, rng, sizes, backward_mask):
    reqs = []
    for n, bwd in zip(sizes, backward_mask):
        idx = rng.integers(0, w.n_pairs, n)
        r = {
            "pg": torch.from_numpy(np.ascontiguousarray(ids[w.pair_geoms[idx]]).astype(np.int32)).pin_memory(),
            "poses": torch.from_numpy(w.poses[idx].copy()).pin_memory(),
            "dims": torch.from_numpy(w.dims[idx].copy()).pin_memory(),
            "tau": torch.from_numpy(w.tau[idx].copy()).pin_memory(),
            "out": torch.empty((n, 8, 8)).pin_memory(),
        }
        if bwd:
            r["gout"] = torch.from_numpy(rng.normal(size=(n, 8, 8)).astype(np.float32)).pin_memory()
            r["gp"] = torch.empty((n, 14)).pin_memory()
            r["gd"] = torch.empty((n, 6)).pin_memory()
        reqs.append(r)
    return reqs


def submit(api, ctx, r):
    return api.cm_submit(ctx, r["pg"], r["poses"], r["out"], r["dims"], r["tau"], r.get("gout"), r.get("gp"),
                         r.get("gd"))


@pytest.fixture(scope="module")
def pool():
    w = synth.config_mixed(n=256, seed=55)
    return w


def test_mixed_requests_match_alone(pool):
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine
    w = pool
    eng = Engine(0, hbm_budget_bytes=8 << 30)
    try:
        ids = eng.add_geometries(w.geoms)
        params = eng.params()
        rng = np.random.default_rng(0)
        sizes = [1, 3, 17, 64, 200, 512, 5, 90, 333, 2, 48, 128] * 2
        reqs = make_requests(w, ids, rng, sizes, [i % 2 == 1 for i in range(len(sizes))])
        api.cm_server_start(eng.ctx, params, max_batch_pairs=1024, n_streams=3)
        tickets = [None] * len(reqs)

        def client(lo):
            for i in range(lo, len(reqs), 3):
                tickets[i] = submit(api, eng.ctx, reqs[i])
        th = [threading.Thread(target=client, args=(k,)) for k in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        peak = 0
        for t in tickets:
            while not api.cm_poll(eng.ctx, t):
                peak = max(peak, api.cm_server_stats(eng.ctx)[2])
            api.cm_wait(eng.ctx, t, 10000)
        pairs, batches, _ = api.cm_server_stats(eng.ctx)
        assert pairs == sum(sizes) and batches >= 2
        assert peak <= 8 << 30
        for r, t in zip(reqs, tickets):
            assert api.cm_request_latency(eng.ctx, t) > 0
            api.cm_release(eng.ctx, t)
        api.cm_server_stop(eng.ctx)
        # each request alone through the direct entry points
        for r in reqs:
            pg, poses, dims, tau = (r[k].cuda() for k in ("pg", "poses", "dims", "tau"))
            alone = eng.forward(pg, poses, dims, tau, params).cpu()
            # the forward's column sums use float atomics (order-dependent rounding): held
            # to the stated parity tolerance, 1e-5
            assert torch.allclose(r["out"], alone, atol=1e-5, rtol=0)
            if "gout" in r:
                # the adjoint sums with atomics: launches agree to FP32 rounding of those sums,
                # held to the gradient tolerance (1e-3 of each pair's largest component)
                gp, gd = eng.backward(pg, poses, dims, tau, r["gout"].cuda(), params)
                got = torch.cat([r["gp"], r["gd"]], 1)
                ref = torch.cat([gp, gd], 1).cpu()
                scale = ref.abs().max(1).values.clamp_min(1e-12)
                assert ((got - ref).abs().max(1).values / scale).max() <= 1e-3
        eng.check()
    finally:
        eng.close()


def test_admission_and_timeouts(pool):
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine
    w = pool
    eng = Engine(0, hbm_budget_bytes=2 << 30)
    try:
        ids = eng.add_geometries(w.geoms)
        params = eng.params()
        api.cm_server_start(eng.ctx, params, max_batch_pairs=8192, n_streams=2)
        rng = np.random.default_rng(1)
        with pytest.raises(api.CMError) as ei:
            api.cm_wait(eng.ctx, 987654, 0)
        assert ei.value.status == api.CM_ERR_NOT_FOUND
        big = make_requests(w, ids, rng, [8192] * 3, [True] * 3)
        tb = [submit(api, eng.ctx, r) for r in big]
        small = make_requests(w, ids, rng, [4], [False])[0]
        ts = submit(api, eng.ctx, small)
        with pytest.raises(api.CMError) as ei:          # still queued behind the big ones
            api.cm_wait(eng.ctx, ts, 0)
        assert ei.value.status == api.CM_ERR_TIMEOUT
        for t in tb + [ts]:
            api.cm_wait(eng.ctx, t, 60000)
        assert np.isfinite(small["out"].numpy()).all()
        api.cm_server_stop(eng.ctx)
        # with a 1 MiB budget: a request that cannot fit even alone is refused at submission,
        # a small one is served
        eng2 = Engine(0, hbm_budget_bytes=1 << 20)
        try:
            ids2 = eng2.add_geometries(w.geoms)
            api.cm_server_start(eng2.ctx, params, max_batch_pairs=8192, n_streams=2)
            huge = make_requests(w, ids2, rng, [8192], [True])[0]
            with pytest.raises(api.CMError) as ei:
                submit(api, eng2.ctx, huge)
            assert ei.value.status == api.CM_ERR_ADMISSION
            tiny = make_requests(w, ids2, rng, [2], [True])[0]
            api.cm_wait(eng2.ctx, submit(api, eng2.ctx, tiny), 60000)
            assert np.isfinite(tiny["gp"].numpy()).all()
            api.cm_server_stop(eng2.ctx)
        finally:
            eng2.close()
    finally:
        eng.close()


def test_single_request_batches_match_alone(pool):
    """Requests submitted one at a time, each waited for before the next, so that every
    batch holds a single request (forward-only and forward+backward, sizes whose buffers
    round differently): results equal the direct entry points' and the admitted bytes
    return to zero."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine
    w = pool
    eng = Engine(0, hbm_budget_bytes=8 << 30)
    try:
        ids = eng.add_geometries(w.geoms)
        params = eng.params()
        rng = np.random.default_rng(1)
        sizes = [1, 2, 3, 7, 16, 63, 64, 65, 100, 257]
        bwd = [i % 2 == 0 for i in range(len(sizes))] + [i % 2 == 1 for i in range(len(sizes))]
        sizes = sizes * 2
        reqs = make_requests(w, ids, rng, sizes, bwd)
        api.cm_server_start(eng.ctx, params, max_batch_pairs=1024, n_streams=2)
        for r in reqs:
            t = submit(api, eng.ctx, r)
            api.cm_wait(eng.ctx, t, 20000)
            api.cm_release(eng.ctx, t)
        pairs, batches, in_use = api.cm_server_stats(eng.ctx)
        assert pairs == sum(sizes) and batches == len(sizes) and in_use == 0
        api.cm_server_stop(eng.ctx)
        for r in reqs:
            pg, poses, dims, tau = (r[k].cuda() for k in ("pg", "poses", "dims", "tau"))
            out = eng.forward(pg, poses, dims, tau, params)
            assert torch.allclose(out.cpu(), r["out"], atol=1e-5, rtol=0)
            if "gout" in r:
                gp, gd = eng.backward(pg, poses, dims, tau, r["gout"].cuda(), params)
                got = torch.cat([r["gp"], r["gd"]], 1)
                ref = torch.cat([gp, gd], 1).cpu()
                scale = ref.abs().max(1).values.clamp_min(1e-12)
                assert ((got - ref).abs().max(1).values / scale).max() <= 1e-3
        eng.check()
    finally:
        eng.close()


def test_admission_by_free_device_memory(pool):
    """Without a budget, admission follows the device's free memory: with most of the GPU
    held elsewhere, a forward+backward request whose batch block (at least 152 scratch
    slices of its largest E_A x E_B at 16 floats, ~290 MB here) exceeds what is free
    fails with CM_ERR_ADMISSION instead of waiting forever, and a small request is still
    served."""
    from paper_2602_20304_gb300 import api
    from paper_2602_20304_gb300.engine import Engine
    w = pool
    nvA, nvB, neA, neB = w.pair_counts()
    big_idx = int(np.argmax(neA * neB))
    assert 152 * int(neA[big_idx] * neB[big_idx]) * 64 > 256 << 20
    eng = Engine(0)
    hog = None
    try:
        ids = eng.add_geometries(w.geoms)
        params = eng.params()
        api.cm_server_start(eng.ctx, params, max_batch_pairs=8192, n_streams=2)
        torch.cuda.synchronize()
        free, _ = torch.cuda.mem_get_info()
        hog = torch.empty(free - (512 << 20), dtype=torch.uint8, device="cuda")   # leave 512 MiB
        rng = np.random.default_rng(3)
        # 512 pairs: a batch gets min(512, CTAs of the launch) >= 152 scratch slices
        ws = w.subset(np.full(512, big_idx))
        big = make_requests(ws, ids, rng, [512], [True])[0]
        t = submit(api, eng.ctx, big)
        with pytest.raises(api.CMError) as ei:
            api.cm_wait(eng.ctx, t, 60000)
        assert ei.value.status == api.CM_ERR_ADMISSION and "free memory" in str(ei.value)
        tiny = make_requests(w, ids, rng, [2], [False])[0]
        api.cm_wait(eng.ctx, submit(api, eng.ctx, tiny), 60000)
        assert np.isfinite(tiny["out"].numpy()).all()
        api.cm_server_stop(eng.ctx)
    finally:
        del hog
        torch.cuda.empty_cache()
        eng.close()
