"""Host logic of the N > 1 paths, on CPU with the gloo backend (world size 2).

Frames are independent once the reference is fixed (Sec. III), so ranks exchange no frame
data: in the bench each tracks its own seeded stream and only the timing is reduced (max
over ranks); a single stream or a camera set is partitioned over the ranks and the records
gathered (``paper_2310_08770_b300.shard``). These tests run the reduction, the partitions
and the gathers as real gloo ranks, without a GPU.
"""
import json
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    from paper_2310_08770_b300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = b.dist_env()
        # per-rank elapsed times: the job's time is the slowest rank's
        elapsed = [3.25, 7.5, 1.0, 2.0][r]
        t_max = b.max_over_ranks(elapsed, w, device="cpu")
        s = synth.frame_stream(seed=b.shard_seed(r), n=64, count=4)
        q.put({"rank": r, "world": w, "t_max": t_max, "seed": b.shard_seed(r),
               "frame_sum": int(s.frames.astype(np.int64).sum()), "ref_sum": float(s.ref.sum())})
        dist.barrier()
    finally:
        dist.destroy_process_group()


REC = np.dtype([("dx", "<f4"), ("dy", "<f4"), ("ipy", "<i4"), ("ipx", "<i4")])


def _track(frames, ref, u):
    """Records of frames against ref. On these CPU ranks the FP64 oracle stands in for each
    rank's GPU tracker: what is under test is the partition and the gather."""
    import oracle
    out = np.zeros(len(frames), REC)
    for i, f in enumerate(frames):
        o = oracle.track_one(np.asarray(f, np.float64), np.asarray(ref, np.float64), u)
        out[i] = (o["dx32"], o["dy32"], o["ipy"], o["ipx"])
    return out


def _cameras():
    from paper_2310_08770_b300 import synth
    cams = []
    for c, N in enumerate((16, 24, 32, 12, 20)):
        rng = np.random.default_rng(100 + c)
        ref = synth.gaussian_spot(N, N, N / 2, N / 2, 1.8, 900.0, 8.0)
        d = rng.uniform(-1.5, 1.5, size=(4, 2))
        fr = np.array([rng.poisson(synth.gaussian_spot(N, N, N / 2 + p[1], N / 2 + p[0], 1.8, 900.0, 8.0))
                       for p in d], np.float64)
        cams.append((ref, fr))
    return cams


def _shard_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2310_08770_b300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = synth.frame_stream(seed=0, n=10_000, count=23)
        lo, hi = shard.frame_range(len(s.frames), world, rank)
        stream = shard.gather_records(_track(s.frames[lo:hi], s.ref, 40), world, rank)
        cams = _cameras()
        owner = shard.camera_ranks(len(cams), world)
        mine = {c: _track(fr, ref, 30) for c, (ref, fr) in enumerate(cams) if owner[c] == rank}
        percam = shard.gather_camera_records(mine, world)
        q.put({"rank": rank, "range": (lo, hi), "stream": stream.tobytes(), "cams": sorted(mine),
               "percam": {k: v.tobytes() for k, v in percam.items()}})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_ranks(world, target=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target or _rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda d: d["rank"])


def test_two_gloo_ranks_reduce_time_and_shard_streams():
    res = _run_ranks(2)
    assert [d["world"] for d in res] == [2, 2]
    # every rank sees the maximum of the per-rank times
    assert all(d["t_max"] == 7.5 for d in res)
    # rank 0 runs the seed-0 workload; the ranks' streams are independent
    assert res[0]["seed"] == 0 and res[1]["seed"] != res[0]["seed"]
    assert res[0]["frame_sum"] != res[1]["frame_sum"]
    # the noise-free reference is the same spot on every rank
    assert res[0]["ref_sum"] == pytest.approx(res[1]["ref_sum"])


def test_two_ranks_partition_a_stream_and_a_camera_set_like_one_rank():
    # frames are independent under a fixed reference: a 23-frame stream split 12 / 11 and five
    # cameras dealt round robin give, gathered, exactly the one-rank records
    from paper_2310_08770_b300 import shard, synth
    res = _run_ranks(2, _shard_main)
    s = synth.frame_stream(seed=0, n=10_000, count=23)
    one = _track(s.frames, s.ref, 40).tobytes()
    assert [d["range"] for d in res] == [(0, 12), (12, 23)]
    assert all(d["stream"] == one for d in res)
    cams = _cameras()
    want = {c: _track(fr, ref, 30).tobytes() for c, (ref, fr) in enumerate(cams)}
    assert res[0]["cams"] == [0, 2, 4] and res[1]["cams"] == [1, 3]
    assert all(d["percam"] == want for d in res)
    # the single-rank forms are the identity
    assert shard.frame_range(23, 1, 0) == (0, 23) and shard.camera_ranks(3, 1) == [0, 0, 0]


def test_frame_ranges_cover_the_stream_once():
    from paper_2310_08770_b300 import shard
    for n in (0, 1, 7, 10_000):
        for world in (1, 2, 3, 8):
            r = [shard.frame_range(n, world, k) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.frame_range(5, 2, 2)


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(4.5, 1) == 4.5


def test_weighted_percentile_counts_frames_not_batches():
    # 39 full batches of 256 frames at 100 us and one 16-frame batch at 10 us:
    # frame-weighted, the short batch does not move p50 or p99
    lat = [100.0] * 39 + [10.0]
    w = [256] * 39 + [16]
    assert bench.weighted_percentile(lat, w, 50) == 100.0
    assert bench.weighted_percentile(lat, w, 99) == 100.0
    # unweighted ordering check on a small case
    assert bench.weighted_percentile([3.0, 1.0, 2.0], [1, 1, 1], 50) == 2.0
    assert bench.weighted_percentile([1.0, 2.0], [1, 3], 50) == 2.0


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 3, 3
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_flop_accounting_matches_folded_formulation():
    # 128 x 128, u = 100: the per-part counts the roofline divides by
    m, h0, wc = 150, 75, 65
    fft = 2 * 2.5 * 128 * 128 * 14
    expect = fft + 6 * 128 * wc + h0 * wc * 64 * 8 + m * m * wc * 2 + (h0 + 1) * wc * 4
    assert bench.flop_per_frame() == expect
    assert bench.grid_size(100) == 150


def test_profile_summary_keys_parse():
    path = bench.PROFILE_FILE
    with open(path) as f:
        kv = dict(line.split(":", 1) for line in f if ":" in line and not line.startswith("#"))
    kv = {k.strip(): v.strip() for k, v in kv.items()}
    assert len(kv["kernel_source_hash"]) == 16
    assert float(kv["dram_bytes_per_launch_full_batch"]) > 256 * 128 * 128 * 2 * 0.99
    json.dumps(kv)
