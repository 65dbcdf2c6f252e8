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


def test_results_identical_alone_and_in_the_mix(cuda_device):
    from paper_1509_00186_b300.serving import run_alone, run_mix
    specs = small_specs()
    summary, outs = run_mix(specs, n_blocks=5, keep_outputs=True)
    assert summary["streams_admitted"] == 4 and summary["seq_gaps"] == 0
    for i, sp in enumerate(specs):
        alone = run_alone(sp, 5)
        assert np.array_equal(outs[i], alone), i


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


def test_sequence_gaps_are_counted_and_repeats_refused(cuda_device):
    import torch
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import Pool, make_block_inputs
    sp = small_specs()[0]
    with Pool(8 << 30, max_streams=2) as pool:
        sid = pool.admit(sp)
        bs = pool.get(sid, "block_samples")
        x = torch.from_numpy(make_block_inputs(sp, bs, 1)).cuda()
        out = torch.empty((sp.n_chan, pool.get(sid, "n_out_per_block")), device="cuda")
        lat = [pool.wait(pool.submit(sid, s, x, out)) for s in (0, 1, 4)]   # blocks 2 and 3 lost
        assert pool.get(sid, "seq_gaps") == 2
        assert all(v >= 0 for v in lat)
        with pytest.raises(cdd.CddError):
            pool.submit(sid, 4, x, out)                       # a repeated block is refused


def test_gsb_and_upgraded_gmrt_mix_meets_the_deadline(cuda_device):
    """Eight streams of the mixed GSB / upgraded-GMRT shapes, arrivals paced at
    20x real time: every block finishes well inside its block duration."""
    from paper_1509_00186_b300.serving import mixed_scenario, run_mix
    summary, _ = run_mix(mixed_scenario(8), n_blocks=4, speedup=20.0)
    assert summary["streams_admitted"] == 8
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
