"""Serving (ccst_server_*): continuous batching of single frames from several cameras of
different sizes. Each result must be the same alone and in the mix; admission refuses
frames when the device slots are full; the load generator accounts for every frame."""
import threading

import numpy as np
import pytest

from paper_2310_08770_b300 import ccst as C
from paper_2310_08770_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08770_b300 import build
    build.build()
    return _t


def cameras(seed=0, sides=(64, 128, 32), n=24):
    rng = np.random.default_rng(seed)
    cams = []
    for N in sides:
        ref = synth.gaussian_spot(N, N, N / 2, N / 2, 3.0, 2000.0, 20.0).astype(np.float32)
        d = rng.uniform(-3, 3, size=(n, 2))
        frames = np.array([rng.poisson(synth.gaussian_spot(N, N, N / 2 + p[0], N / 2 + p[1], 3.0, 2000.0, 20.0))
                           for p in d]).astype(np.uint16)
        cams.append((ref, frames))
    return cams


def make_server(cams, slots=64, max_batch=64):
    t = C.Tracker(cams[0][0], upsample=100, in_dtype="u16")
    ids = [0] + [C.ccst_add_reference(t.ctx, ref, *ref.shape) for ref, _ in cams[1:]]
    srv = C.ccst_server_create(t.ctx, slots, max_batch)
    return t, ids, srv


def submit_wait(srv, ref_id, frame):
    while True:
        try:
            return C.ccst_server_submit(srv, ref_id, frame)
        except C.CcstError as e:
            if e.code != C.E_BUSY:
                raise


def test_each_result_is_the_same_alone_and_in_the_mix(torch):
    cams = cameras()
    t, ids, srv = make_server(cams)
    try:
        alone = {}
        for k, (_, frames) in enumerate(cams):
            for i in range(len(frames)):
                tk = C.ccst_server_submit(srv, ids[k], frames[i])
                alone[(k, i)] = C.ccst_server_poll(srv, tk, 5_000_000).tobytes()
        # the mix: three client threads, one per camera, each frame submitted three times
        got = {}
        lock = threading.Lock()

        def client(k):
            frames = cams[k][1]
            tickets = [(i, submit_wait(srv, ids[k], frames[i])) for _ in range(3) for i in range(len(frames))]
            for i, tk in tickets:
                r = C.ccst_server_poll(srv, tk, 5_000_000)
                with lock:
                    got.setdefault((k, i), []).append(r.tobytes())
        th = [threading.Thread(target=client, args=(k,)) for k in range(len(cams))]
        for x in th:
            x.start()
        for x in th:
            x.join()
        assert set(got) == set(alone)
        for key, rs in got.items():
            assert len(rs) == 3 and all(r == alone[key] for r in rs), key
        st = C.ccst_server_read_stats(srv)
        assert st["completed"] == st["submitted"] and st["in_flight"] == 0
        assert st["mean_batch"] > 1.0                  # the mix was batched
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_result_equals_the_context_path(torch):
    cams = cameras(seed=1, sides=(64, 128), n=6)
    t, ids, srv = make_server(cams)
    try:
        for k, (ref, frames) in enumerate(cams):
            single = C.Tracker(ref, upsample=100, in_dtype="u16", max_batch=len(frames))
            out = single.empty_results(len(frames))
            C.ccst_track(single.ctx, torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16),
                         len(frames), 0, out)
            C.ccst_sync(single.ctx)
            want = C.decode(out)
            single.close()
            for i in range(len(frames)):
                r = C.ccst_server_poll(srv, C.ccst_server_submit(srv, ids[k], frames[i]), 5_000_000)
                assert r.tobytes() == want[i].tobytes()
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_admission_refuses_when_slots_are_full(torch):
    cams = cameras(seed=2, sides=(128,), n=8)
    t, ids, srv = make_server(cams, slots=2, max_batch=2)
    try:
        tickets, refused = [], 0
        for i in range(400):
            try:
                tickets.append(C.ccst_server_submit(srv, 0, cams[0][1][i % 8]))
            except C.CcstError as e:
                assert e.code == C.E_BUSY
                refused += 1
        for tk in tickets:
            assert C.ccst_server_poll(srv, tk, 5_000_000) is not None
        st = C.ccst_server_read_stats(srv)
        assert refused > 0 and st["rejected"] == refused and st["completed"] == len(tickets)
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_loadgen_accounts_for_every_frame(torch):
    cams = cameras(seed=3, sides=(64, 128, 32), n=16)
    t, ids, srv = make_server(cams, slots=256, max_batch=256)
    try:
        st = C.ccst_server_loadgen(srv, ids, [2000.0, 5000.0, 10000.0], [f for _, f in cams], 0.3, seed=4)
        assert st["in_flight"] == 0 and st["completed"] == st["submitted"] and st["submitted"] > 3000
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_server_errors(torch):
    cams = cameras(seed=5, sides=(32,), n=2)
    t, ids, srv = make_server(cams, slots=4, max_batch=4)
    try:
        with pytest.raises(C.CcstError):
            C.ccst_server_submit(srv, 9, cams[0][1][0])          # unknown camera
        with pytest.raises(C.CcstError):
            C.ccst_server_poll(srv, 123456, 10)                   # unknown ticket
        tk = C.ccst_server_submit(srv, 0, cams[0][1][0])
        assert C.ccst_server_poll(srv, tk, 5_000_000) is not None
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_general_size_cameras_equal_the_roi_path(torch):
    # the first camera (96 px) makes a general-shape context; 48 and 192 px cameras take the
    # general-size kernel too, 64 px the power-of-two kernel, all in the same batches
    cams = cameras(seed=9, sides=(96, 64, 48, 192), n=8)
    t, ids, srv = make_server(cams)
    try:
        want = {}
        for k, (_, frames) in enumerate(cams):
            d = torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
            out = t.empty_results(len(frames))
            C.ccst_track_rois(t.ctx, C.make_rois([d[i] for i in range(len(frames))], [ids[k]] * len(frames)),
                              len(frames), out)
            C.ccst_sync(t.ctx)
            for i, r in enumerate(C.decode(out)):
                assert bool(r["flags"] & (C.R_GENERIC | C.R_FP32_GENERAL)) == (frames.shape[-1] != 64)
                want[(k, i)] = r.tobytes()
        tickets = [((k, i), submit_wait(srv, ids[k], cams[k][1][i])) for i in range(8) for k in range(len(cams))]
        for key, tk in tickets:
            assert C.ccst_server_poll(srv, tk, 20_000_000).tobytes() == want[key], key
        st = C.ccst_server_read_stats(srv)
        assert st["completed"] == st["submitted"] and st["in_flight"] == 0
        # the load generator over the same cameras accounts for every frame
        st = C.ccst_server_loadgen(srv, ids, [500.0, 2000.0, 1000.0, 200.0], [f for _, f in cams], 0.2, seed=3)
        assert st["in_flight"] == 0 and st["completed"] == st["submitted"] > 0
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_double_float_cameras_beside_fp32_and_power_of_two_ones(torch):
    # a 40 px camera (no FP32 plan: the double-float kernel, on the batch's second stream
    # after the FP32 launches), 96 px (FP32 general-size) and 64 / 128 px (power-of-two) in
    # the same batches: every result equals the ROI path's for that frame
    cams = cameras(seed=13, sides=(64, 40, 96, 128), n=6)
    t, ids, srv = make_server(cams)
    try:
        want = {}
        for k, (_, frames) in enumerate(cams):
            d = torch.from_numpy(frames.view(np.int16)).cuda().view(torch.uint16)
            out = t.empty_results(len(frames))
            C.ccst_track_rois(t.ctx, C.make_rois([d[i] for i in range(len(frames))], [ids[k]] * len(frames)),
                              len(frames), out)
            C.ccst_sync(t.ctx)
            for i, r in enumerate(C.decode(out)):
                if frames.shape[-1] == 40:
                    assert r["flags"] & C.R_GENERIC and not r["flags"] & C.R_FP32_GENERAL
                want[(k, i)] = r.tobytes()
        tickets = [((k, i), submit_wait(srv, ids[k], cams[k][1][i])) for i in range(6) for k in range(len(cams))]
        for key, tk in tickets:
            assert C.ccst_server_poll(srv, tk, 20_000_000).tobytes() == want[key], key
        st = C.ccst_server_read_stats(srv)
        assert st["completed"] == st["submitted"] and st["in_flight"] == 0
    finally:
        C.ccst_server_destroy(srv)
        t.close()


def test_admission_by_bytes_charges_each_frame_its_own_size(torch):
    # a budget of one 128 x 128 uint16 frame (32 KiB): a 128 px frame alone fills it, while up
    # to 16 frames of a 32 px camera (2 KiB each) fit at once; nothing larger than the budget
    # is ever admissible
    cams = cameras(seed=11, sides=(128, 32), n=8)
    t = C.Tracker(cams[0][0], upsample=100, in_dtype="u16")
    ids = [0, C.ccst_add_reference(t.ctx, cams[1][0], 32, 32)]
    srv = C.ccst_server_create_ex(t.ctx, 64, 2, 128 * 128 * 2)
    try:
        admitted, refused = 0, 0
        for i in range(3000):
            k = 1 if i % 10 else 0
            try:
                C.ccst_server_submit(srv, ids[k], cams[k][1][i % 8], keep=False)
                admitted += 1
            except C.CcstError as e:
                assert e.code == C.E_BUSY
                refused += 1
        for _ in range(200000):
            st = C.ccst_server_read_stats(srv)
            if st["in_flight"] == 0:
                break
        assert st["completed"] == admitted and st["rejected"] == refused and refused > 0
        assert st["budget_bytes"] == 32768 and 2048 < st["max_bytes_in_flight"] <= 32768
        assert st["bytes_in_flight"] == 0
    finally:
        C.ccst_server_destroy(srv)
    small = C.ccst_server_create_ex(t.ctx, 8, 1, 16 * 1024)      # below one 128 px frame
    try:
        with pytest.raises(C.CcstError) as e:
            C.ccst_server_submit(small, 0, cams[0][1][0])
        assert e.value.code == C.E_INVALID
        tk = C.ccst_server_submit(small, ids[1], cams[1][1][0])
        assert C.ccst_server_poll(small, tk, 5_000_000) is not None
    finally:
        C.ccst_server_destroy(small)
    for bad in [(0, 1, 1 << 20), (4, 0, 1 << 20), (4, 5, 1 << 20), (4, 1, 100)]:
        with pytest.raises(C.CcstError):
            C.ccst_server_create_ex(t.ctx, *bad)
    t.close()


def test_plain_configuration_launches_one_frame_at_a_time(torch):
    cams = cameras(seed=12, sides=(64, 128), n=10)
    t = C.Tracker(cams[0][0], upsample=100, in_dtype="u16")
    ids = [0, C.ccst_add_reference(t.ctx, cams[1][0], 128, 128)]
    batched = C.ccst_server_create_ex(t.ctx, 256, 4, 8 << 20)
    plain = C.ccst_server_create_ex(t.ctx, 1, 1, 8 << 20)
    try:
        want = {}
        for k in range(2):
            for i in range(10):
                want[(k, i)] = C.ccst_server_poll(batched, C.ccst_server_submit(batched, ids[k], cams[k][1][i]),
                                                  5_000_000).tobytes()
        tickets = [((k, i), C.ccst_server_submit(plain, ids[k], cams[k][1][i])) for i in range(10) for k in range(2)]
        for key, tk in tickets:
            assert C.ccst_server_poll(plain, tk, 5_000_000).tobytes() == want[key]
        st = C.ccst_server_read_stats(plain)
        assert st["completed"] == 20 and st["batches"] == 20 and st["mean_batch"] == 1.0
    finally:
        C.ccst_server_destroy(batched)
        C.ccst_server_destroy(plain)
        t.close()
