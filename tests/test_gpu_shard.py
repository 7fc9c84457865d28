"""Aux shards on the device: two DF handles holding the B rows [0, P) and
[P, Naux) of (H2O)_3, built one after the other on one GPU.  Their partial
J and K add up to the whole tensor's, in FP64 to 1e-10 (the two paths share
the integrals but not the triangular solve's blocking), and in split FP16 to
the mixed build's own error (each shard takes its own scales).  Shard rows
equal the corresponding rows of the whole B; the SCF and MP2 refuse a
shard, and direct mode has none."""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


def test_shards_sum_to_whole(gpu_ctx):
    import torch
    import paper_2502_17963_gb300 as bqc
    from paper_2502_17963_gb300 import shard
    mol = workload.water_cluster(3)
    basis = bqc.Basis(gpu_ctx, mol)
    whole = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16)
    rng = np.random.default_rng(31)
    C = torch.tensor(np.linalg.qr(rng.standard_normal((basis.nbf, basis.nocc)))[0] * 0.5,
                     device="cuda")
    J, K = whole.jk(C, bqc.PREC_FP64)
    J16, K16 = whole.jk(C, bqc.PREC_MIXED_F16X3)
    B = whole.copy(0)
    ranges = shard.aux_ranges(basis.naux, 2)
    Js, Ks, J16s, K16s = 0, 0, 0, 0
    for p0, p1 in ranges:
        d = bqc.DF(gpu_ctx, basis, keep_fp32=bqc.SHADOW_F16, aux_range=(p0, p1))
        assert d.aux_range == (p0, p1)
        Bs = d.copy(0)
        assert Bs.shape[0] == p1 - p0
        assert (Bs - B[p0:p1]).abs().max().item() < 1e-11
        j, k = d.jk(C, bqc.PREC_FP64)
        Js, Ks = Js + j, Ks + k
        j, k = d.jk(C, bqc.PREC_MIXED_F16X3)
        J16s, K16s = J16s + j, K16s + k
        with pytest.raises(bqc.BqcError):
            bqc.scf_run(gpu_ctx, d)
        d.close()
    dJ, dK = (Js - J).abs().max().item(), (Ks - K).abs().max().item()
    d16 = max((J16s - J).abs().max().item(), (K16s - K).abs().max().item())
    dw = max((J16 - J).abs().max().item(), (K16 - K).abs().max().item())
    print(f"shards FP64: max|dJ| {dJ:.2e} max|dK| {dK:.2e}; F16X3 vs FP64: sharded {d16:.2e}, "
          f"whole {dw:.2e}")
    assert dJ < 1e-10 and dK < 1e-10
    assert d16 < 10 * dw + 1e-9
    with pytest.raises(bqc.BqcError) as e:
        bqc.DF(gpu_ctx, basis, mode=bqc.DF_DIRECT, aux_range=(0, 10))
    assert e.value.status == -9
    with pytest.raises(bqc.BqcError) as e:
        bqc.DF(gpu_ctx, basis, aux_range=(10, basis.naux + 1))
    assert e.value.status == -1
