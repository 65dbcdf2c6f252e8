"""Serving pool: admission by HBM budget, overlapping streams, sequence gaps,
and each stream's result the same alone and in the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def small_specs():
    from paper_1509_00186_b300.serving import StreamSpec
    return [StreamSpec(325.0, 2.0, 32, 20.0, block_seconds=0.1, seed=1),
            StreamSpec(610.0, 4.0, 64, 80.0, block_seconds=0.1, seed=2),
            StreamSpec(650.0, 12.5, 128, 35.0, block_seconds=0.1, seed=3),
            StreamSpec(325.0, 4.0, 64, 120.0, block_seconds=0.1, seed=4)]


@pytest.mark.parametrize("host", [True, False])
def test_results_identical_alone_and_in_the_mix(cuda_device, host):
    """Four streams served together (host-buffer or device-buffer ingest) give,
    block for block, the bits each gives alone through a plain plan."""
    from paper_1509_00186_b300.serving import run_alone, run_mix
    specs = small_specs()
    summary, outs = run_mix(specs, n_blocks=5, keep_outputs=True, host=host)
    assert summary["admitted_at_once"] == 4 and summary["blocks"] == 20
    for i, sp in enumerate(specs):
        alone = run_alone(sp, 5)
        assert np.array_equal(outs[i], alone), i


def test_streams_admitted_mid_run_from_the_queue(cuda_device):
    """A budget that holds only two of the four streams: the others wait in
    the pool's queue and are admitted while the run goes on, as earlier
    streams finish and are released.  Every stream's output is still the
    same, bit for bit, as its run alone."""
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import run_alone, run_mix
    specs = small_specs()
    need = []
    for sp in specs:
        n = sp.n_fft()
        with cdd.Plan(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, n, sp.n_avg,
                      segments_per_block=sp.segments_per_block(n)) as p:
            need.append(p.get("bytes_needed") + p.get("host_staging_bytes"))
    budget = sorted(need)[-1] + sorted(need)[-2]
    assert budget < sum(need)
    summary, outs = run_mix(specs, n_blocks=4, keep_outputs=True, budget_bytes=budget,
                            stagger_blocks=0.0)
    assert summary["admitted_from_queue"] >= 1
    assert summary["admitted_at_once"] + summary["admitted_from_queue"] == 4
    for i, sp in enumerate(specs):
        assert np.array_equal(outs[i], run_alone(sp, 4)), i


def test_admission_respects_the_hbm_budget(cuda_device):
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import Pool
    specs = small_specs()
    need = []
    for sp in specs:
        with cdd.Plan(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, sp.n_fft(), sp.n_avg) as p:
            need.append(p.get("bytes_needed"))
    budget = need[0] + need[1] + max(need[2], need[3]) // 2     # room for two of them
    with Pool(budget, max_streams=8) as pool:
        a = pool.admit(specs[0])
        b = pool.admit(specs[1])
        assert pool.used_bytes() <= budget
        with pytest.raises(cdd.CddError) as ei:
            pool.admit(specs[2])
        assert ei.value.code == cdd.CDD_EBUSY
        pool.release(a)                                       # memory frees up: admitted now
        c = pool.admit(specs[0])
        assert c >= 0 and pool.used_bytes() <= budget
        pool.release(b)
        pool.release(c)
        assert pool.used_bytes() == 0


def test_gaps_are_refused_until_resync(cuda_device):
    """Blocks must come in order: a repeated block and a block after a gap
    are refused (nothing enqueued).  cdd_pool_stream_resync moves the stream
    past the loss, counts the skipped blocks and restarts it from zero
    history, so the next block's output is a fresh stream's."""
    import torch
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import Pool, make_block_inputs
    sp = small_specs()[0]
    with Pool(8 << 30, max_streams=2) as pool:
        sid = pool.admit(sp)
        bs = pool.get(sid, "block_samples")
        n_out = pool.get(sid, "n_out_per_block")
        x = torch.from_numpy(make_block_inputs(sp, bs, 5)).cuda()
        out = torch.empty((5, sp.n_chan, n_out), device="cuda")
        for b in (0, 1):
            assert pool.wait(pool.submit(sid, b, x[b * bs:(b + 1) * bs], out[b])) >= 0
        for bad in (1, 4):                                    # repeated; after a gap
            with pytest.raises(cdd.CddError) as ei:
                pool.submit(sid, bad, x[4 * bs:], out[4])
            assert ei.value.code == cdd.CDD_EINVAL
        assert pool.get(sid, "seq_gaps") == 0
        pool.resync(sid, 4)                                   # blocks 2 and 3 were lost
        assert pool.get(sid, "seq_gaps") == 2
        pool.wait(pool.submit(sid, 4, x[4 * bs:], out[4]))
        n = sp.n_fft()
        with cdd.Plan(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, n, sp.n_avg,
                      segments_per_block=sp.segments_per_block(n)) as fresh:
            want = fresh.execute(x[4 * bs:])
        assert torch.equal(out[4], want)


def test_latency_runs_from_the_block_arrival(cuda_device):
    """A block that arrived 50 ms before its submission reports at least 50 ms;
    host-buffer submission is refused for a stream admitted without host
    staging."""
    import torch
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import Pool, make_block_inputs
    sp = small_specs()[1]
    with Pool(8 << 30, max_streams=2) as pool:
        sid = pool.admit(sp)
        bs = pool.get(sid, "block_samples")
        x = torch.from_numpy(make_block_inputs(sp, bs, 1)).cuda()
        out = torch.empty((sp.n_chan, pool.get(sid, "n_out_per_block")), device="cuda")
        lat = pool.wait(pool.submit(sid, 0, x, out, t_arrival_ms=cdd.cdd_pool_clock_ms() - 50.0))
        assert lat >= 50.0
        lat = pool.wait(pool.submit(sid, 1, x, out))
        assert 0.0 <= lat < 50.0
        with pytest.raises(cdd.CddError) as ei:
            pool.submit(sid, 2, x.cpu().pin_memory(), out.cpu().pin_memory())
        assert ei.value.code == cdd.CDD_ESTATE


def test_many_blocks_in_one_call_equal_one_by_one(cuda_device):
    """cdd_pool_submit_many enqueues blocks of several streams in one call;
    the outputs equal the blocks submitted one by one."""
    import torch
    from paper_1509_00186_b300.serving import Pool, make_block_inputs, run_alone
    specs = small_specs()[:2]
    with Pool(8 << 30, max_streams=2) as pool:
        sids = [pool.admit(sp, host=True) for sp in specs]
        xs, outs = [], []
        for sp, sid in zip(specs, sids):
            bs = pool.get(sid, "block_samples")
            xs.append(torch.from_numpy(make_block_inputs(sp, bs, 3)).pin_memory())
            outs.append(torch.empty((3, sp.n_chan, pool.get(sid, "n_out_per_block"))).pin_memory())
        blocks = []
        for b in range(3):
            for j, sid in enumerate(sids):
                bs = pool.get(sid, "block_samples")
                blocks.append((sid, b, xs[j][b * bs:(b + 1) * bs], outs[j][b], None))
        from paper_1509_00186_b300 import cdd
        now = cdd.cdd_pool_clock_ms()
        tickets = pool.submit_many([blk[:4] + (now,) for blk in blocks], host=True)
        assert all(pool.wait(t) >= 0 for t in tickets)
    for j, sp in enumerate(specs):
        assert np.array_equal(outs[j].numpy(), run_alone(sp, 3))


def test_gsb_and_upgraded_gmrt_mix_meets_the_deadline(cuda_device):
    """Eight streams of the mixed GSB / upgraded-GMRT shapes from pinned host
    buffers, arrivals paced at 20x real time: every block, copies included,
    finishes inside its paced deadline (block duration / 20) counted from
    its arrival."""
    from paper_1509_00186_b300.serving import mixed_scenario, run_mix
    summary, _ = run_mix(mixed_scenario(8), n_blocks=4, speedup=20.0)
    assert summary["admitted_at_once"] + summary["admitted_from_queue"] == 8
    assert summary["missed_deadlines"] == 0
    assert summary["latency_ms"]["p99"] < summary["deadline_ms"]["min"] / 20


def test_stream_moves_to_another_pool(cuda_device):
    """A stream checkpointed after three blocks (state and next sequence number)
    and imported into a stream of another pool continues bit for bit: its
    outputs equal those of the stream run without interruption."""
    import torch
    from paper_1509_00186_b300.serving import Pool, make_block_inputs, run_alone
    sp = small_specs()[1]
    n_blocks = 6
    want = run_alone(sp, n_blocks)
    with Pool(8 << 30, max_streams=2) as first, Pool(8 << 30, max_streams=2) as second:
        a = first.admit(sp)
        bs = first.get(a, "block_samples")
        n_out = first.get(a, "n_out_per_block")
        x = torch.from_numpy(make_block_inputs(sp, bs, n_blocks)).cuda()
        outs = torch.empty((n_blocks, sp.n_chan, n_out), device="cuda")
        for b in range(3):
            first.wait(first.submit(a, b, x[b * bs:(b + 1) * bs], outs[b]))
        state, seq = first.export_stream(a)
        assert seq == 3
        first.release(a)
        c = second.admit(sp)
        second.import_stream(c, state, seq)
        for b in range(3, n_blocks):
            second.wait(second.submit(c, b, x[b * bs:(b + 1) * bs], outs[b]))
        assert second.get(c, "seq_gaps") == 0
        assert np.array_equal(outs.cpu().numpy(), want)


def test_pool_checkpoint_refusals(cuda_device):
    """Pool checkpoints refuse unknown streams and negative sequence numbers."""
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import Pool
    with Pool(1 << 30, max_streams=2) as pool:
        with pytest.raises(cdd.CddError) as ei:
            pool.export_stream(0)
        assert ei.value.code == cdd.CDD_EINVAL
        sid = pool.admit(small_specs()[0])
        state, seq = pool.export_stream(sid)
        for bad_sid, bad_seq in ((1, 0), (sid, -1)):
            with pytest.raises(cdd.CddError) as ei:
                pool.import_stream(bad_sid, state, bad_seq)
            assert ei.value.code == cdd.CDD_EINVAL
