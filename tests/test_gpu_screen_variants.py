"""The three survivor compactions of the screened three-centre integrals
(bqc_int3c_screened): the library's sorted prefix, the paper's per-warp loop
buffer (Algorithm 1) and the two-kernel global index list compute the same
triplets with the same arithmetic, so their outputs must be bitwise equal,
over windows of aux functions that start and end inside shells, with strong
screening (tau = 1e-6, most triplets skipped) and the benchmark's 1e-10."""
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
        for v in (1, 2):
            assert torch.equal(outs[v], outs[0]), (name, tau, p0, p1, v)
    # and the sorted-prefix window equals the raw integrals of bqc_int3c at the same tau
    full = bqc.int3c(basis, schwarz=tau)
    assert torch.equal(df.int3c_screened(0, basis.naux, 0), full)
    print(f"{name} tau {tau:g}: kept {kept}/{cand} = {kept / cand:.3f}")
