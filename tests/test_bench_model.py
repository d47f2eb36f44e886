"""The benchmark's algorithmic model (the bytes and flops behind its roofline and per-iteration figures),
checked against the per-launch figures stated for the 128^3 / k = 32 / p = 8 workload: K1 moves A + 2nk
values when the recomputed rho is formed in K3 (FP64, 2 <= p <= 16, warp-chunk layout), A + 3nk otherwise;
one FP64 iteration moves A + 11 nk * 8 bytes."""
import pytest

import bench

N, K, P = 128 ** 3, 32, 8
Z = 7 * 128 ** 3 - 6 * 128 ** 2
A64 = 12.0 * Z + 8.0 * (N + 1)


@pytest.mark.parametrize("k,p,prec,expect", [
    (32, 8, "fp64", True), (32, 16, "fp64", True), (32, 2, "fp64", True), (32, 1, "fp64", False),
    (32, 32, "fp64", False), (64, 8, "fp64", True), (256, 16, "fp64", True), (24, 8, "fp64", False),
    (6, 3, "fp64", False), (5, 5, "fp64", False), (16, 4, "fp64", True), (32, 8, "fp32_refine", False),
])
def test_rho_in_k3_rule(k, p, prec, expect):
    assert bench.rho_in_k3(k, p, prec) is expect


def test_model_of_the_bench_workload():
    m = bench.kernel_model(N, K, P, Z, 8, A64, rho_k3=True)
    nk8 = N * K * 8
    assert m["op_gram"]["bytes"] == pytest.approx(A64 + 2 * nk8)
    assert m["update_xr"]["bytes"] == pytest.approx(6 * nk8) == pytest.approx(3.221225472e9)
    assert m["update_p"]["bytes"] == pytest.approx(3 * nk8)
    total = sum(v["bytes"] for v in m.values())
    assert total == pytest.approx(A64 + 11 * nk8) and total == pytest.approx(6.097e9, rel=1e-3)
    # FP64-pipe work: BOP 2kz, the two BAXPYs of K2 4npk, K3's 2npk
    assert m["op_gram"]["alu"] == pytest.approx(0.93323264e9)
    assert m["update_xr"]["alu"] == pytest.approx(2.147483648e9)
    assert m["update_p"]["alu"] == pytest.approx(1.073741824e9)
    # the Dot2 block products total 6 npk + 2 nk wherever the recomputed rho is formed
    dot2 = sum(v["gram"] for v in m.values())
    assert dot2 == pytest.approx(sum(v["gram"] for v in bench.kernel_model(N, K, P, Z, 8, A64).values()))
    assert dot2 == pytest.approx(6 * N * P * K + 2 * N * K)
    # recomputed rho in K1: one more pass over R there
    m1 = bench.kernel_model(N, K, P, Z, 8, A64, rho_k3=False)
    assert sum(v["bytes"] for v in m1.values()) == pytest.approx(A64 + 12 * nk8)
