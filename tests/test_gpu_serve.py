"""Serving: continuous batching of independent SCF solves on one GPU.

Each result must be the same alone (one slot, one request at a time) and in
the mix (four slots, all requests in flight together); the kernels are
deterministic (no atomics in the reductions), so the FP64 energies agree to
rounding and the mixed ones to the same.  Also: solves actually overlap,
admission rejects a request larger than the budget, and a solve that hits
max_iter reports BQC_E_NOT_CONVERGED.
"""
import pytest

import oracle
import workload

pytestmark = pytest.mark.gpu

MOLS = ["h2o", "w2", "w3", "w4", "w5", "w6"]


@pytest.fixture(scope="module")
def bqc():
    import paper_2502_17963_gb300 as m
    return m


def _run(bqc, ctx, names, slots, prec, budget=0):
    srv = bqc.Server(ctx, max_slots=slots, prec=prec, hbm_budget=budget)
    out = {}
    if slots == 1:
        for n in names:
            t = srv.submit(workload.molecule_for(n))
            srv.drain(600)
            out[n] = srv.poll(t)
    else:
        ts = {n: srv.submit(workload.molecule_for(n)) for n in names}
        srv.drain(600)
        out = {n: srv.poll(t) for n, t in ts.items()}
    srv.close()
    return out


@pytest.mark.parametrize("prec", [0, 2])
def test_alone_equals_mix(gpu_ctx, bqc, prec):
    alone = _run(bqc, gpu_ctx, MOLS, 1, prec, budget=8 << 30)
    mix = _run(bqc, gpu_ctx, MOLS, 4, prec, budget=8 << 30)
    for n in MOLS:
        a, m = alone[n], mix[n]
        assert a["status"] == 0 and m["status"] == 0, (n, a, m)
        assert abs(a["energy"] - m["energy"]) <= 1e-10, (n, a["energy"], m["energy"])
    # solves overlapped: some request was admitted before another finished
    spans = sorted((r["t_admit"], r["t_done"]) for r in mix.values())
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    # and the energies are the oracle's
    for n in ["h2o", "w2"]:
        mol = workload.molecule_for(n)
        I = oracle.system_integrals(mol)
        B, _ = oracle.df_tensor(I["aux"], I["orb"])
        ro = oracle.rhf(I["S"], I["H"], lambda C: oracle.jk_df(B, C), mol.nocc, I["enuc"])
        assert abs(mix[n]["energy"] - ro.energy) < 1e-8


def test_admission_rejects_oversized(gpu_ctx, bqc):
    srv = bqc.Server(gpu_ctx, max_slots=1, hbm_budget=256 << 20)
    with pytest.raises(bqc.BqcError) as e:
        srv.submit(workload.water_cluster(16))
    assert e.value.status == -3
    srv.close()


def test_not_converged_status(gpu_ctx, bqc):
    srv = bqc.Server(gpu_ctx, max_slots=1, max_iter=2, prec=0, hbm_budget=1 << 30)
    t = srv.submit(workload.water_cluster(2))
    srv.drain(300)
    r = srv.poll(t)
    assert r["status"] == -4 and r["iterations"] == 2
    srv.close()
