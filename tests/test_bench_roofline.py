"""Host arithmetic of the bench line's roofline (no GPU): the dominant
kernel's achieved rate is the method's FP64 work (Grams n q (q+1) each, two
per iteration; update 2 n q^2) over the product kernel's time, the BF16 pipe
figure counts the digit-pair products the emulation issues (15 per Gram
product at five digits, 21 per update product), and the traffic figures are
per launch, with the algorithmic bytes of the digit slices read once."""
import pytest

import bench


def solve_info(ms_tc=300.0, sizes=(1_000_000, 31_623, 1000), iters=(8, 13, 0), q=750):
    one = {"q": q, "sizes": list(sizes), "iters": list(iters), "ritz_calls": 21, "solve_flops": 3.4e12,
           "ms_tc_product": ms_tc}
    for k in ("galerkin", "coarse", "prolong", "factor", "spmm", "gram", "ritz", "update", "residual"):
        one["ms_" + k] = 10.0
    one["ms_solve"] = 500.0
    return one


def test_method_work_over_product_time():
    info = solve_info()
    top = bench.roofline(info, [info], None, 500, {"bf16_tflops_sustained": 1700.0}, "measured", "mixed", 1e-5)
    n0, n1, q = 1_000_000, 31_623, 750
    gram = 8 * 2.0 * n0 * q * (q + 1) + 13 * 2.0 * n1 * q * (q + 1)
    upd = 8 * 2.0 * n0 * q * q + 13 * 2.0 * n1 * q * q
    assert top["achieved"] == pytest.approx((gram + upd) / 0.300 / 1e12, rel=1e-12)
    assert top["frac"] == pytest.approx(top["achieved"] / 1700.0, rel=1e-12)
    # five digits per Gram value at tol 1e-5: 15 digit-pair products; 21 for the update
    assert top["bf16_pipe"]["achieved"] == pytest.approx((15 * gram + 21 * upd) / 0.300 / 1e12, rel=1e-12)
    assert top["launches_per_step"] == 3 * (8 + 13)


def test_six_digit_grams_below_1e6():
    info = solve_info()
    top = bench.roofline(info, [info], None, 500, {"bf16_tflops_sustained": 1700.0}, "measured", "mixed", 1e-7)
    assert "21 (Grams)" in top["bf16_pipe"]["note"]


def test_traffic_per_launch_and_algorithmic_bytes():
    # one level, one iteration: three launches (two Grams, one update)
    n, q = 200_000, 750
    tr = bench.tc_traffic([n, 1000], [1, 0], q, gram_digits=5)
    qp = 768  # columns padded to 32
    gram_alg = 2 * (5 * 2.0) * n * qp  # both operands' five BF16 slices
    upd_alg = 6 * 2.0 * n * qp + 8.0 * n * q  # six slices of Psi, FP64 output
    assert tr["algorithmic_per_launch"] == pytest.approx((2 * gram_alg + upd_alg) / 3, rel=1e-12)
    # the captures at 200,000 rows themselves
    per_row = bench.TC_TRAFFIC_PER_ROW
    assert tr["per_launch"] == pytest.approx((2 * per_row["gram"] + per_row["update"]) * n / 3, rel=1e-12)
    # the captured update reads its slices about once
    assert per_row["update"] * n / upd_alg == pytest.approx(1.0, abs=0.02)
