"""The three survivor compactions of the screened three-centre integrals
(bqc_int3c_screened): the library's sorted prefix, the paper's per-warp loop
buffer (Algorithm 1) and the two-kernel global index list compute the same
triplets with the same recursion, over windows of aux functions that start
and end inside shells, with strong screening (tau = 1e-6 and 1e-4, most
triplets skipped) and the benchmark's 1e-10.  The index-list kernel compiles
to the same arithmetic as the sorted prefix's and must be bitwise equal; the
loop-buffer kernel inlines the recursion into a different loop, where the
compiler contracts some products into FMAs differently, so its values may
differ in the last bit (measured up to 1e-15): it must agree to 1e-14
absolute, and a missing or doubled triplet would be an O(1e-2..1) error."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,tau", [("w3", 1e-6), ("w16", 1e-10), ("w16", 1e-4)])
def test_variants_bitwise_equal(gpu_ctx, name, tau):
    import torch
    import paper_2502_17963_gb300 as bqc
    mol = workload.molecule_for(name)
    basis = bqc.Basis(gpu_ctx, mol)
    df = bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, schwarz=tau, keep_fp32=False)
    cand, kept = df.screening()
    for p0, p1 in ((0, basis.naux), (7, basis.naux // 2 + 5)):
        outs = [df.int3c_screened(p0, p1, v) for v in range(3)]
        torch.cuda.synchronize()
        assert outs[0].abs().max().item() > 0.0
        assert torch.equal(outs[2], outs[0]), (name, tau, p0, p1)
        d1 = (outs[1] - outs[0]).abs().max().item()
        assert d1 < 1e-14, (name, tau, p0, p1, d1)
    # and the sorted-prefix window equals the raw integrals of bqc_int3c at the same tau
    full = bqc.int3c(basis, schwarz=tau)
    assert torch.equal(df.int3c_screened(0, basis.naux, 0), full)
    print(f"{name} tau {tau:g}: kept {kept}/{cand} = {kept / cand:.3f}")
