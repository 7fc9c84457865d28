"""Grouped split-FP16 Fock builds of independent molecules (serving batches).

The grouped launches run every molecule's X pass, FP64 J pass and SYRK with
that molecule's own plan, so K must equal the single-molecule build bit for
bit (the same tiles, chains and aux chunks) and J to the rounding of the J
pass's aux chunking (the single build streams J in pipeline pieces).  Sizes
mix tile widths (nocc 5 .. 80, so per-problem xn 32 .. 96 in one launch) and
ragged 128-row tails; more than twelve handles exercise the split into
several launches.  A grouped server must give the same energies as the
per-stream server.
"""
import numpy as np
import pytest

import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


def _handles(bqc, ctx, names):
    out = []
    for nm in names:
        basis = bqc.Basis(ctx, workload.molecule_for(nm))
        out.append(bqc.DF(ctx, basis, keep_fp32=bqc.SHADOW_F16))
    return out


def _orbitals(n, nocc, seed):
    import torch
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((n, nocc)) * (1.0 / np.sqrt(n))
    return torch.tensor(C, device="cuda")


@pytest.mark.parametrize("names", [["w3", "w8", "w16", "h2o"], ["h2o"] * 13 + ["w5"]])
def test_grouped_equals_single(gpu_ctx, bqc, names):
    import torch
    dfs = _handles(bqc, gpu_ctx, names)
    Cs = [_orbitals(d.basis.nbf, d.basis.nocc, 100 + i) for i, d in enumerate(dfs)]
    ref = [d.jk(C, bqc.PREC_MIXED_F16X3) for d, C in zip(dfs, Cs)]
    Js, Ks = bqc.jk_grouped(dfs, Cs)
    torch.cuda.synchronize()
    for (J1, K1), J2, K2, nm in zip(ref, Js, Ks, names):
        assert torch.equal(K1, K2), (nm, float((K1 - K2).abs().max()), float(K1.abs().max()))
        # J: float-float sums (~2^-46 per term) over a different aux
        # chunking; J cancels by up to ~100x against its terms here
        ja = float(J1.abs().max())
        assert float((J1 - J2).abs().max()) <= 1e-11 * ja, nm
        assert torch.equal(J2, J2.T) and torch.equal(K2, K2.T)
    # repeat: the grouped build leaves nothing behind that changes the next
    Js2, Ks2 = bqc.jk_grouped(dfs, Cs)
    for a, b in zip(Ks, Ks2):
        assert torch.equal(a, b)
    for a, b in zip(Js, Js2):
        assert torch.equal(a, b)
    for d in dfs:
        d.close()


def test_grouped_rejects(gpu_ctx, bqc):
    mol = workload.molecule_for("w2")
    b = bqc.Basis(gpu_ctx, mol)
    d16 = bqc.DF(gpu_ctx, b, keep_fp32=bqc.SHADOW_F16)
    d32 = bqc.DF(gpu_ctx, b, keep_fp32=bqc.SHADOW_TF32)
    C = _orbitals(b.nbf, b.nocc, 7)
    with pytest.raises(bqc.BqcError) as e:
        bqc.jk_grouped([d16, d32], [C, C])
    assert e.value.status == bqc.BQC_E_UNSUPPORTED
    with pytest.raises(bqc.BqcError) as e:
        bqc.jk_grouped([d16, d16], [C, C])
    assert e.value.status == bqc.BQC_E_INVALID
    d16.close()
    d32.close()


def test_grouped_server_equals_per_stream(gpu_ctx, bqc):
    names = ["h2o", "w2", "w3", "w4", "w5", "w6"]

    def run(grouped):
        srv = bqc.Server(gpu_ctx, max_slots=4, prec=bqc.PREC_MIXED_F16X3, hbm_budget=8 << 30,
                         grouped=grouped, group_window_us=2000.0)
        ts = {n: srv.submit(workload.molecule_for(n)) for n in names}
        srv.drain(600)
        out = {n: srv.poll(t) for n, t in ts.items()}
        st = srv.group_stats()
        srv.close()
        return out, st

    per, st0 = run(False)
    grp, st1 = run(True)
    assert st0 == dict(batches=0, builds=0, max_batch=0)
    for n in names:
        a, g = per[n], grp[n]
        assert a["status"] == 0 and g["status"] == 0, (n, a, g)
        # both finish on FP64 builds: the energies agree to the SCF tolerance
        assert abs(a["energy"] - g["energy"]) <= 1e-8, (n, a["energy"], g["energy"])
    mixed = sum(r["iterations_mixed"] for r in grp.values())
    assert st1["builds"] >= mixed > 0
    assert 1 <= st1["max_batch"] <= 4 and st1["batches"] <= st1["builds"]
    print("grouped server:", st1, "mixed iterations", mixed)
