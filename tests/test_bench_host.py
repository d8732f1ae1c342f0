"""Host logic of bench.py: the algorithmic byte counts and the multi-rank timing (replicas on
two gloo ranks on the CPU; no GPU)."""
import os
import socket
import time

import pytest

import bench


def test_full_transform_moves_every_cell_four_times():
    # z = n = L: both passes of Algorithm 1 read and write all L cells; Algorithm 2 likewise
    for l in (2, 5, 8, 16):
        L = 1 << l
        assert bench.alg_cells_tft(l, L, L) == 4 * L
        assert bench.alg_cells_itft(l, L, L) == 4 * L


def test_truncated_counts():
    # L = 2^16, n = z = 40000: 157 partial-height rows of 256 cells after the column pass
    l, n = 16, 40000
    assert bench.alg_cells_tft(l, n, n) == n + 157 * 256 + 157 * 256 + n
    # counts never exceed the full transform and grow with n
    prev = 0
    for n in (1, 2, 255, 256, 257, 32769, 40000, 65535, 65536):
        c = bench.alg_cells_tft(l, n, n)
        assert prev <= c <= 4 * 65536
        prev = c
        assert bench.alg_cells_itft(l, n, n) <= 4 * 65536


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    ws, r = bench.dist_init("gloo")
    delay = 0.05 * (rank + 1)
    secs = bench.timed_steps(lambda: time.sleep(delay), steps=3, warmup=3, sync=lambda: None)
    out.put((r, ws, secs))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in procs]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    res.sort()
    assert [r for r, _, _ in res] == [0, 1] and all(ws == 2 for _, ws, _ in res)
    # both ranks report the same (slowest) time, at least rank 1's 3 x 0.1 s
    assert abs(res[0][2] - res[1][2]) < 1e-9
    assert res[0][2] >= 0.3


def test_clock_samples_count_only_inside_the_timed_region(monkeypatch):
    """The sampler keeps the samples stamped between the region's start and its end plus one
    interval, and reports a throttle reason only if one of those samples shows it."""
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)

    def line(mhz, hw="Not Active", pcap="Not Active"):
        return f"0, {mhz}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pcap}"

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.ClockSampler(0)
    c.proc = FakeProc()
    c.lines = [(0.0, line(1500, hw="Active")), (1.00, line(2070)), (1.04, line(2055, pcap="Active")),
               (1.20, line(900))]
    c.t0, c.t1 = 0.99, 1.05
    out = c.stop()
    assert out["samples"] == 2 and out["sm_mhz"] == (2070 + 2055) / 2
    assert out["reasons"] == ["sw_power_cap"] and "note" not in out
    # a region shorter than the interval: the first sample after its start, flagged
    c.lines = [(0.0, line(1500)), (2.5, line(2070))]
    c.t0, c.t1 = 2.0, 2.01
    out = c.stop()
    assert out["samples"] == 1 and out["sm_mhz"] == 2070 and "note" in out


def test_cell_stride_defaults_to_aligned_cells_and_checks_requests():
    assert bench.cell_stride(513, 0) == 514  # W = 513 at N = 32768: 16-byte aligned cells
    assert bench.cell_stride(17, 0) == 18
    assert bench.cell_stride(513, 528) == 528  # 128-byte aligned cells
    for bad in (512, 515):
        with pytest.raises(SystemExit):
            bench.cell_stride(513, bad)


def test_plan_bytes_of_the_benchmark_tft():
    """The l = 16, n = 40000 TFT's jobs read and write 2.0x the algorithmic bytes of the
    paper's two-pass schedule: four passes of 16-cell jobs, each cell read and written once a
    pass (the first pass reads the n inputs, the others about n cells)."""
    import paper_0810_3203_gb300 as tg
    tg.load()
    b = bench.plan_bytes(tg, 0, 16, 40000, 32768)
    alg = bench.alg_cells_tft(16, 40000, 40000) * bench.cell_bytes(32768)
    # reads 40000 + 40960 + 40192 + 40000 cells, writes 40960 + 40192 + 40000 + 40000
    assert b == 2 * 161152 * bench.cell_bytes(32768)
    assert 1.95 < b / alg < 2.05


def test_reference_steps_stay_bounded():
    """The reference arm's oracle work stays near 25 round trips at n = 40000 for any step
    count, and keeps n = 40000 for short runs."""
    assert bench.reference_sample_n(1, 3) == 40000
    assert bench.reference_sample_n(22, 3) == 40000
    for steps in (30, 100, 400):
        n = bench.reference_sample_n(steps, 3)
        assert 2048 <= n < 40000 and (steps + 3) * n <= 25 * 40000
    assert bench.reference_sample_n(1000, 3) == 2048  # the floor
