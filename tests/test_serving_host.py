"""Host logic of the serving driver (CPU): each stream's transform length.
A stream takes the library's Sec. 2.3 rule (n_fft = 0: the smallest power of
two above twice the lowest channel's smear) raised to at least 2048; the
oracle's geometry and the C library must both accept it."""
import numpy as np

import oracle as O


def test_stream_transform_length_is_the_smallest_fit_and_a_valid_plan():
    from paper_1509_00186_b300 import cdd
    from paper_1509_00186_b300.serving import StreamSpec, mixed_scenario
    specs = mixed_scenario(40, seed=3) + [StreamSpec(325.0, 32.0, 512, 150.0),
                                          StreamSpec(150.0, 16.0, 256, 150.0),
                                          StreamSpec(650.0, 200.0, 2048, 5.0)]
    seen = set()
    for sp in specs:
        n = sp.n_fft()
        g = O.plan_geometry(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, n, sp.n_avg)
        floor = max(2048.0, 2.0 * g.n_disp + 1e-9)
        assert n & (n - 1) == 0 and n >= floor and (n == 2048 or n // 2 <= 2.0 * g.n_disp)
        assert g.n_ov < n
        p = cdd.cdd_plan_create(sp.f_center_mhz, sp.bandwidth_mhz, sp.n_chan, sp.dm, n, sp.n_avg)
        try:
            assert cdd.cdd_plan_get(p, "n_fft") == n
            assert cdd.cdd_plan_get(p, "n_ov") == g.n_ov
        finally:
            cdd.cdd_destroy(p)
        seen.add(n)
    assert len(seen) >= 2                 # the cases span more than one transform length
    assert np.all([sp.dm >= 5.0 and sp.dm <= 150.0 for sp in specs[:40]])
