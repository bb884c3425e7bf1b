"""Host-side helpers of bench.py: the guarded extras and the algorithmic work
counts that the roofline fractions divide by."""
import bench


def test_a_failing_extra_reports_its_error_instead_of_raising():
    def boom():
        raise RuntimeError("no device")
    assert bench.guarded("extra", boom) == {"extra": {"error": "RuntimeError: no device"}}
    assert bench.guarded("extra", lambda a: {"extra": a}, 3) == {"extra": 3}


def test_lifted_flops_on_a_hand_counted_element():
    """n = 1, p = 1, Radau K = 3: interior 3, element block 3 + 2 + 1 = 6.
    Collocation rows have 3 + 1 + 1 = 5 nonzeros: 3 rows x 5 x 6 = 90 flops of
    rank-1 updates; the continuity row (2 nonzeros) 1 x 2 x 3 = 6; Cholesky of
    3 columns of an order-6 block: 5 x 6 + 4 x 5 + 3 x 4 = 62."""
    assert bench.lifted_flops(1, 1, 1, 3) == 90 + 6 + 62
    assert bench.lifted_flops(1, 1, 7, 3) == 7 * (90 + 6 + 62)
    # Gauss K = 4: continuity rows touch all 5 points and the next z_0 (6 nonzeros)
    kn, me = 4, 4 + 2 + 1
    chol = sum((me - c - 1) * (me - c) for c in range(kn))
    assert bench.lifted_flops(1, 1, 1, 4, gauss=True) == kn * 6 * 7 + 1 * 6 * 7 + chol
