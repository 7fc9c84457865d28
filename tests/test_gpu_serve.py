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


def _sampled_requests(count=20, nmax=6):
    """The first `count` requests of the seed-2025 Poisson stream with n <= nmax
    (geometry seed = request id), as (name, Molecule)."""
    out = []
    for _, n, rid in workload.serving_stream(nreq=2000):
        if n <= nmax:
            out.append((f"r{rid}", workload.water_cluster(n, seed=rid)))
        if len(out) == count:
            break
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (2, 1e-8)])
def test_alone_equals_mix_sampled_stream(gpu_ctx, bqc, prec, tol):
    reqs = _sampled_requests()
    assert len(reqs) == 20 and len({len(m.Z) for _, m in reqs}) > 2
    srv = bqc.Server(gpu_ctx, max_slots=1, prec=prec, hbm_budget=8 << 30)
    alone = {}
    for name, mol in reqs:
        t = srv.submit(mol)
        srv.drain(600)
        alone[name] = srv.poll(t)
    srv.close()
    srv = bqc.Server(gpu_ctx, max_slots=6, prec=prec, hbm_budget=8 << 30)
    ts = {name: srv.submit(mol) for name, mol in reqs}
    srv.drain(900)
    mix = {name: srv.poll(t) for name, t in ts.items()}
    srv.close()
    for name, _ in reqs:
        a, m = alone[name], mix[name]
        assert a["status"] == 0 and m["status"] == 0, (name, a, m)
        assert abs(a["energy"] - m["energy"]) <= tol, (name, a["energy"], m["energy"])
        assert a["iterations"] == m["iterations"]
    spans = sorted((r["t_admit"], r["t_done"]) for r in mix.values())
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


@pytest.mark.parametrize("policy", [0, 1])
def test_backfill_admission_and_priority(gpu_ctx, bqc, policy):
    big, small = workload.water_cluster(6), workload.single_water()
    fb = bqc.serve_footprint(150, 450, 30, prec=2)
    fs = bqc.serve_footprint(26, 92, 5, prec=2)
    assert fs < fb
    # two large requests never fit together, a large and a small one do
    srv = bqc.Server(gpu_ctx, max_slots=3, prec=2, hbm_budget=2 * fb - 1, policy=policy)
    t1, t2, t3 = srv.submit(big), srv.submit(big), srv.submit(small)
    srv.drain(600)
    r1, r2, r3 = srv.poll(t1), srv.poll(t2), srv.poll(t3)
    srv.close()
    assert r1["status"] == 0 and r2["status"] == 0 and r3["status"] == 0
    assert r1["energy"] == r2["energy"]
    if policy == bqc.SERVE_BACKFILL:
        # the small request was admitted past the waiting large one, at a higher priority
        assert r3["t_admit"] < r2["t_admit"]
        assert r3["priority"] <= r1["priority"]
    else:
        assert r3["t_admit"] >= r2["t_admit"]
        assert r3["priority"] == r1["priority"] == r2["priority"]


def test_cancel_queued_and_running(gpu_ctx, bqc):
    """A queued request cancelled completes at once with BQC_E_CANCELLED; a
    running one stops at its next step boundary with the same status; the
    server keeps serving, and a done request is left as it is."""
    import time
    srv = bqc.Server(gpu_ctx, max_slots=1, prec=bqc.PREC_FP64, hbm_budget=4 << 30)
    t_run = srv.submit(workload.water_cluster(16))
    t_q = srv.submit(workload.molecule_for("w2"))
    t_ok = srv.submit(workload.molecule_for("h2o"))
    srv.cancel(t_q)
    r_q = srv.poll(t_q)
    assert r_q is not None and r_q["status"] == bqc.BQC_E_CANCELLED
    time.sleep(0.3)  # the first solve is admitted (one slot) and running
    srv.cancel(t_run)
    srv.drain(300)
    r_run, r_ok = srv.poll(t_run), srv.poll(t_ok)
    assert r_run["status"] == bqc.BQC_E_CANCELLED, r_run
    assert r_ok["status"] == 0, r_ok
    srv.cancel(t_ok)  # already done: unchanged
    assert srv.poll(t_ok)["status"] == 0
    with pytest.raises(bqc.BqcError) as e:
        srv.cancel(123456789)
    assert e.value.status == bqc.BQC_E_INVALID
    srv.close()
