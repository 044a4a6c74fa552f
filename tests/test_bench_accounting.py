"""The roofline accounting of bench.py on the CPU: the algorithmic bytes and flops of one
tensor-core preconditioner launch on the 128^2 workload (BF16 inverse 16 x 1152^2 x 2 B, residual
image 16 x 1152 x 64 x 2 B, z written and r read in FP32), and the tiling bench.py assumes equals
the one the library launches (sg_plan_query) for every workload and batch instance that uses it."""
import pytest

import bench
import sg_workloads as w

SG_MIXED = 1


def test_product_bytes_and_flops_on_the_bench_workload():
    p = w.config("ricker128")
    assert bench.tc_product_shape(p) == (33, 16, 1152, 32)
    assert bench.tc_product_bytes(p) == 16 * 1152 ** 2 * 2 + 16 * 1152 * 64 * 2 + 2 * 16 * 33 ** 2 * 20 * 4
    assert bench.tc_product_bytes(p) == 47_614_464
    assert bench.tc_product_flops(p) == 2 * 16 * 1152 ** 2 * 64 == 2_717_908_992


def test_bench_tiling_equals_the_library_plan():
    from paper_2512_23027_gb300 import build as b
    b.build()
    from paper_2512_23027_gb300.binding import plan_query
    n = 0
    for prob in [w.config("ricker128"), w.config("small"), w.config("pulse32")] + w.batch_problems(64):
        plan = plan_query(prob, SG_MIXED)
        if not plan["mma"]:
            continue
        L, nsub, Kp, NB = bench.tc_product_shape(prob)
        assert (L, nsub, Kp, NB) == (plan["L"], plan["nsub"], plan["mma_kp"], plan["mma_nb"])
        n += 1
    assert n >= 20
