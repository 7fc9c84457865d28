"""Host-side pieces that need no GPU: the seeded input generators and the
binding's marshalling of a molecule into the C ABI's request struct."""
import ctypes

import numpy as np

import workload


def test_cluster_sizes_and_determinism():
    for n, (N, naux, nocc) in {1: (25, 75, 5), 32: (800, 2400, 160), 64: (1600, 4800, 320),
                               128: (3200, 9600, 640)}.items():
        m = workload.water_cluster(n)
        nf = lambda sh: sum((s.l + 1) * (s.l + 2) // 2 for s in sh)
        assert (nf(m.orb), nf(m.aux), m.nocc) == (N, naux, nocc)
        assert len(m.Z) == 3 * n and m.xyz.shape == (3 * n, 3)
    a, b = workload.water_cluster(16), workload.water_cluster(16)
    assert np.array_equal(a.xyz, b.xyz)
    c = workload.water_cluster(16, seed=17)
    assert not np.array_equal(a.xyz, c.xyz)
    # single water: the config-1 basis (O 6s4p, H 4s; aux O 6s6p6d, H 4s4p)
    w = workload.single_water()
    nf = lambda sh: sum((s.l + 1) * (s.l + 2) // 2 for s in sh)
    assert (nf(w.orb), nf(w.aux), w.nocc) == (26, 92, 5)


def test_geometry_is_physical():
    m = workload.water_cluster(64)
    xyz = m.xyz.reshape(64, 3, 3)
    # O-H 0.9572 A and the HOH angle 104.52 deg in every monomer (bohr here)
    a0 = 0.529177210903
    for w in xyz:
        d1, d2 = np.linalg.norm(w[1] - w[0]), np.linalg.norm(w[2] - w[0])
        assert abs(d1 * a0 - 0.9572) < 1e-9 and abs(d2 * a0 - 0.9572) < 1e-9
        cosang = np.dot(w[1] - w[0], w[2] - w[0]) / (d1 * d2)
        assert abs(np.degrees(np.arccos(cosang)) - 104.52) < 1e-7


def test_serving_stream_seeded():
    s1, s2 = workload.serving_stream(nreq=100), workload.serving_stream(nreq=100)
    assert s1 == s2
    t = [x[0] for x in s1]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert all(2 <= x[1] <= 48 for x in s1) and [x[2] for x in s1] == list(range(100))
    assert 2.0 < t[-1] < 10.0  # mean gap 50 ms


def test_molecule_request_marshalling():
    import paper_2502_17963_gb300 as bqc
    m = workload.water_cluster(2)
    req, keep = bqc.molecule_request(m)
    assert req.natom == 6 and req.norb_shell == len(m.orb) and req.naux_shell == len(m.aux)
    assert [req.Z[i] for i in range(6)] == [int(z) for z in m.Z]
    assert np.allclose([req.xyz_bohr[i] for i in range(18)], m.xyz.reshape(-1))
    for k, s in enumerate(m.orb):
        e = req.orb[k]
        assert (e.atom, e.l, e.nprim) == (s.atom, s.l, len(s.exps))
        assert [e.exps[i] for i in range(e.nprim)] == list(s.exps)
        assert [e.coefs[i] for i in range(e.nprim)] == list(s.coefs)
    assert ctypes.sizeof(bqc.bqc_shell) == 32
