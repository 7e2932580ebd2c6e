"""The stoichiometry-product microbenchmark (bode_stoich_bench): both forms
of f = N r -- the sparse FP32 scatter of the generated integrators and the
warp-level TF32 tensor-core product with the rates split into two TF32
words -- against an FP64 evaluation on the benchmark network.  Errors are
relative to each species' sum of |terms| over every reactant and product
occurrence (the scale at which FP32 sums round): the sparse form <= 1e-6,
the two-word TF32 form (each rate to ~2^-22, then FP32 accumulation of the
products) <= 1e-5."""
import pytest

from paper_1611_02274_gb300 import binding as B
from paper_1611_02274_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [0, 1])
def test_stoich_product_forms_against_fp64(variant):
    w = W.massaction(nsys=8, seed=0)
    h = B.register_workload(w)
    try:
        ms, err = B.stoich_bench(h, variant, 4096, 3)
        assert ms > 0.0
        assert err <= (1e-6 if variant == 0 else 1e-5), err
    finally:
        B.release(h)


def test_stoich_bench_arguments():
    w = W.vdp(8)
    h = B.register_workload(w)
    try:
        with pytest.raises(B.BatchOdeError) as e:
            B.stoich_bench(h, 0, 4096, 1)
        assert e.value.code == B.ODE_ERR_ARG
    finally:
        B.release(h)
    w = W.massaction(nsys=8, seed=0)
    h = B.register_workload(w)
    try:
        for bad in ((2, 4096, 1), (0, 100, 1), (0, 4096, -1)):
            with pytest.raises(B.BatchOdeError) as e:
                B.stoich_bench(h, *bad)
            assert e.value.code == B.ODE_ERR_ARG
    finally:
        B.release(h)
