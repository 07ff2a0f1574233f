"""GPU parity of libgcamps against the FP64 oracle, through the C ABI.

Bars (fixed before measuring):
* tableau (forward and inverse), Weyl strings, bond dimensions, disentangler decisions:
  bit-exact / identical;
* state vector (d^n <= 6561): relative 2-norm error <= 1e-10 after the best global phase
  (a Clifford given by its generator images has no defined global phase);
* <W> for Weyl strings, Schmidt values: absolute error <= 1e-10.
"""
import numpy as np
import pytest

from oracle import clifford, statevector as sv
from oracle.gcamps import GCAMPS
from oracle.weyl import Weyl
from synth import brickwork_circuit, t_gate_phases

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    return G


def oracle_run(gates, n, d, chi_max, cutoff, max_sweeps=8):
    g = GCAMPS(n, d, chi_max=chi_max, cutoff=cutoff, max_sweeps=max_sweeps)
    for gt in gates:
        g.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            g.disentangle()
    return g


def gpu_run(G, gates, n, d, chi_max, cutoff, max_sweeps=8, cluster_size=8):
    sim = G.Simulator(n, d, chi_max=chi_max, cutoff=cutoff, max_sweeps=max_sweeps, cluster_size=cluster_size)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    return sim


def inverse_exps(tab):
    rows = tab.inverse_rows()
    n = tab.n
    e = np.zeros((2 * n, 2 * n), dtype=np.uint8)
    p = np.zeros(2 * n, dtype=np.uint8)
    for k, w in enumerate(rows):
        e[k, :n] = w.x
        e[k, n:] = w.z
        p[k] = w.r
    return e, p


def assert_same_tableaux(sim, ref):
    e, p = sim.tableau()
    re_, rp = ref.tab.exps_phase()
    assert np.array_equal(e, re_)
    assert np.array_equal(p, rp)
    ie, ip = sim.inverse_tableau()
    rie, rip = inverse_exps(ref.tab)
    assert np.array_equal(ie, rie)
    assert np.array_equal(ip, rip)


@pytest.mark.parametrize("d,n,seed", [(2, 6, 1), (3, 5, 2), (3, 9, 3), (2, 13, 4)])
def test_clifford_only_tableau_bit_exact(G, d, n, seed):
    gates = brickwork_circuit(n, d, 2 * n, 0, seed)
    sim = gpu_run(G, gates, n, d, 8, 1e-12)
    ref = oracle_run(gates, n, d, 8, 1e-12)
    assert_same_tableaux(sim, ref)
    assert sim.stats()["clifford_gates"] == len(gates)


@pytest.mark.parametrize("d", [2, 3])
def test_single_qudit_cliffords(G, d):
    n = 4
    sim = G.Simulator(n, d, chi_max=8)
    ref = GCAMPS(n, d, chi_max=8)
    rng = np.random.default_rng(d)
    one = [clifford.H_gate(d), clifford.S_gate(d)]
    for step in range(30):
        if step % 3 == 2:
            gates = brickwork_circuit(n, d, 1, 0, 50 + step)
            for g in gates:
                sim.apply_clifford(g.q0, g.q1, G.sp4_images(d, g.sp_index, g.shift))
                ref.apply_gate(g)
            continue
        u = one[rng.integers(2)]
        q = int(rng.integers(n))
        imgs = clifford.images_by_conjugation(u, 1, d)
        flat = [int(imgs[0].x[0]), int(imgs[0].z[0]), imgs[0].r, int(imgs[1].x[0]), int(imgs[1].z[0]), imgs[1].r]
        sim.apply_clifford(q, -1, flat)
        ref.apply_clifford([q], imgs)
    sim.sync()
    assert_same_tableaux(sim, ref)


@pytest.mark.parametrize("d,n,seed", [(2, 8, 7), (3, 8, 8)])
def test_weyl_string_of_t_gate(G, d, n, seed):
    """P = C^dag Z_k C from the inverse-tableau row vs Gaussian elimination (Sec. 2.3.1)."""
    gates = brickwork_circuit(n, d, n, 0, seed)
    sim = G.Simulator(n, d, chi_max=32, max_sweeps=0)
    sim.run(G.ops_from_gates(gates, d))
    ref = GCAMPS(n, d, chi_max=32)
    for g in gates:
        ref.apply_gate(g)
    for k in range(n):
        want = ref.weyl_of_z(k)
        sim.apply_nonclifford(k, [0.0] * d)   # identity gate: only the Weyl string is recorded
        r, x, z = sim.last_weyl()
        assert r == want.r and np.array_equal(x, want.x) and np.array_equal(z, want.z), k


@pytest.mark.parametrize("d,n,layers,t,seed", [(3, 8, 8, 8, 1), (3, 8, 8, 8, 2), (2, 8, 8, 8, 1),
                                               (3, 6, 10, 12, 3), (2, 10, 10, 10, 5)])
def test_small_circuits_vs_dense_and_oracle(G, d, n, layers, t, seed):
    gates = brickwork_circuit(n, d, layers, t, seed)
    sim = gpu_run(G, gates, n, d, 64, 1e-14)
    ref = oracle_run(gates, n, d, 64, 1e-14)
    assert sim.decisions() == ref.decisions
    assert sim.bond_dims() == ref.mps.bond_dims()
    assert_same_tableaux(sim, ref)
    psi = sv.run(gates, n, d)
    err, _ = sv.same_up_to_phase(sim.statevector(), psi)
    assert err < TOL
    rng = np.random.default_rng(seed)
    for _ in range(5):
        x, z = rng.integers(0, d, n), rng.integers(0, d, n)
        want = sv.expect_weyl(psi, Weyl(0, x, z, d), n, d)
        assert abs(sim.expect_weyl(x, z) - want) < TOL
    z0 = np.zeros(n, dtype=np.int64)
    z0[0] = 1
    assert abs(sim.expect_weyl(np.zeros(n, dtype=np.int64), z0) - sv.expect_weyl(psi, Weyl(0, np.zeros(n), z0, d), n, d)) < TOL
    st = sim.stats()
    assert st["t_gates"] == t and st["status"] == 0
    assert st["candidates_scored"] == ref.candidates_scored


def test_config1_full_amplitudes(G):
    """Plain FP64, qutrits, n = 8, 8 layers, 8 T gates, chi_max = 64, no truncation: the full
    6561-amplitude vector and <Z_0> against dense simulation."""
    d, n = 3, 8
    gates = brickwork_circuit(n, d, 8, 8, 1)
    sim = gpu_run(G, gates, n, d, 64, 1e-14)
    psi = sv.run(gates, n, d)
    v = sim.statevector()
    err, ph = sv.same_up_to_phase(v, psi)
    assert err < TOL
    for y in (0, 1, 100, 3280, 6560):
        digits = [(y // d ** (n - 1 - j)) % d for j in range(n)]
        assert abs(sim.amplitude(digits) * ph - psi[y]) < TOL


def test_no_disentangling_exact_and_chi_growth(G):
    d, n = 3, 6
    gates = brickwork_circuit(n, d, 6, 6, 4)
    sim = gpu_run(G, gates, n, d, 243, 1e-14, max_sweeps=0)
    ref = oracle_run(gates, n, d, 243, 1e-14, max_sweeps=0)
    assert sim.bond_dims() == ref.mps.bond_dims()
    assert max(sim.bond_dims()) > 3
    err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
    assert err < TOL


def test_truncation_matches_oracle(G):
    """chi_max binds (d = 3, chi_max = 3): both sides truncate the same way."""
    d, n = 3, 7
    gates = brickwork_circuit(n, d, 7, 10, 6)
    sim = gpu_run(G, gates, n, d, 3, 1e-12, max_sweeps=0)
    ref = oracle_run(gates, n, d, 3, 1e-12, max_sweeps=0)
    assert sim.bond_dims() == ref.mps.bond_dims()
    assert max(sim.bond_dims()) == 3
    err, _ = sv.same_up_to_phase(sim.statevector(), ref.statevector())
    assert err < 1e-9
    assert abs(sim.stats()["discarded_weight"] - ref.discarded) < 1e-10


@pytest.mark.parametrize("d,seed", [(3, 1), (2, 1), (2, 5), (3, 8)])
def test_full_size_benchmark_circuit(G, d, seed):
    """Circuits of the benchmark workload (n = 32, 24 layers, 32 T gates, chi_max = 256, cutoff
    1e-12): every decision, the tableaux, bond dimensions, Schmidt values and <W> against the
    oracle run of the same circuit.  Qubit seed 5 has a near-tie between two classes that a
    cancelled Householder tail decided wrongly; qutrit seed 8 runs a QR sweep into subnormal
    pivots after an MPO whose support spans 31 sites."""
    n, layers, t, chi, cut = 32, 24, 32, 256, 1e-12
    gates = brickwork_circuit(n, d, layers, t, seed)
    sim = gpu_run(G, gates, n, d, chi, cut)
    ref = oracle_run(gates, n, d, chi, cut)
    assert sim.decisions() == ref.decisions
    assert sim.bond_dims() == ref.mps.bond_dims()
    assert_same_tableaux(sim, ref)
    for b in range(0, n - 1, 5):
        s = sim.schmidt_values(b)
        s = s[s > 1e-13]
        want = ref.mps.schmidt_values(b)
        want = want[want > 1e-13]
        assert len(s) == len(want) and np.max(np.abs(s - want)) < TOL
    rng = np.random.default_rng(d)
    for _ in range(4):
        x, z = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64)
        sites = rng.choice(n, 3, replace=False)
        x[sites] = rng.integers(0, d, 3)
        z[sites] = rng.integers(0, d, 3)
        assert abs(sim.expect_weyl(x, z) - ref.expect_weyl(x, z)) < TOL
    st = sim.stats()
    assert st["t_gates"] == t and st["candidates_scored"] == ref.candidates_scored


def test_batch_matches_single_runs(G):
    d, n = 3, 10
    circuits = [brickwork_circuit(n, d, 8, 10, s) for s in (11, 12, 13)]
    ops = [G.ops_from_gates(c, d) for c in circuits]
    begin = np.cumsum([0] + [len(o) for o in ops]).astype(np.int32)
    sim = G.Simulator(n, d, chi_max=32, cutoff=1e-12, batch=3)
    sim.run(np.concatenate(ops), begin)
    sim.sync()
    for c, gates in enumerate(circuits):
        ref = oracle_run(gates, n, d, 32, 1e-12)
        assert sim.decisions(c) == ref.decisions
        e, p = sim.tableau(c)
        re_, rp = ref.tab.exps_phase()
        assert np.array_equal(e, re_) and np.array_equal(p, rp)
        assert sim.bond_dims(c) == ref.mps.bond_dims()


def test_invalid_input_leaves_handle_usable(G):
    d, n = 3, 4
    sim = G.Simulator(n, d, chi_max=8)
    bad = np.array(G.sp4_images(d, 5, (0, 0, 0, 0)))
    bad[0] = (bad[0] + 1) % d                         # breaks the symplectic form
    with pytest.raises(G.GcampsError) as ei:
        sim.apply_clifford(0, 1, bad)
    assert ei.value.code == 1
    with pytest.raises(G.GcampsError):
        sim.apply_clifford(0, 0, G.sp4_images(d, 5, (0, 0, 0, 0)))
    with pytest.raises(G.GcampsError):
        sim.apply_nonclifford(n, t_gate_phases(d))
    odd_phase = np.array(G.sp4_images(d, 5, (0, 0, 0, 0)))
    odd_phase[4] = 1                                   # tau^1 is not a power of omega for d = 3
    with pytest.raises(G.GcampsError):
        sim.apply_clifford(0, 1, odd_phase)
    sim.apply_clifford(0, 1, G.sp4_images(d, 5, (1, 0, 0, 2)))
    sim.apply_nonclifford(1, t_gate_phases(d))
    sim.disentangle()
    sim.sync()
    assert sim.stats()["status"] == 0


def test_reset(G):
    d, n = 3, 6
    gates = brickwork_circuit(n, d, 6, 6, 21)
    sim = gpu_run(G, gates, n, d, 32, 1e-12)
    sim.reset()
    e, p = sim.tableau()
    assert np.array_equal(e, GCAMPS(n, d, 8).tab.exps_phase()[0]) and not p.any()
    assert sim.bond_dims() == [1] * (n - 1)
    assert sim.stats()["t_gates"] == 0
    sim.run(G.ops_from_gates(gates, d))
    ref = oracle_run(gates, n, d, 32, 1e-12)
    assert sim.decisions() == ref.decisions


@pytest.mark.parametrize("csize", [1, 2, 4, 12, 14, 16])
def test_cluster_sizes_give_identical_decisions(G, csize):
    """The disentangler decisions do not depend on how many CTAs score the classes (qutrits,
    n = 12, chi up to 27, where the Renyi-2 pruning path is taken)."""
    d, n = 3, 12
    gates = brickwork_circuit(n, d, 12, 16, 31)
    sim = gpu_run(G, gates, n, d, 64, 1e-12, cluster_size=csize)
    ref = oracle_run(gates, n, d, 64, 1e-12)
    assert sim.decisions() == ref.decisions
    assert sim.bond_dims() == ref.mps.bond_dims()
    st = sim.stats()
    assert st["vn_evaluations"] <= st["candidates_scored"]


@pytest.mark.parametrize("min_m", [0, 100])
def test_exact_evaluations_on_ctas_or_warps_give_oracle_decisions(G, min_m):
    """Exact class evaluations at warp-level sizes (m <= 27) run one per CTA (min_m = 0: every short
    exact list) or one per warp (min_m = 100): either way the decisions, bond dimensions and Schmidt values
    are the oracle's (qutrits, n = 12, chi up to 27, 16-CTA clusters)."""
    d, n = 3, 12
    gates = brickwork_circuit(n, d, 12, 16, 31)
    sim = G.Simulator(n, d, chi_max=64, cutoff=1e-12, max_sweeps=8, cluster_size=16)
    sim.set_exact_cta(min_m)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    ref = oracle_run(gates, n, d, 64, 1e-12)
    assert sim.decisions() == ref.decisions
    assert sim.bond_dims() == ref.mps.bond_dims()
    for b in range(n - 1):
        s = sim.schmidt_values(b)
        s = s[s > 1e-13]
        want = ref.mps.schmidt_values(b)
        want = want[want > 1e-13]
        assert len(s) == len(want) and np.max(np.abs(s - want)) < TOL
    with pytest.raises(G.GcampsError):
        sim.set_exact_cta(-1)


def test_renyi2_pruning_is_exact_on_large_bonds(G):
    """Bonds with Gram size > 9 use the Renyi-2 bound: decisions still equal the oracle's, which
    scores every class by SVD."""
    d, n = 3, 8
    gates = brickwork_circuit(n, d, 10, 14, 41)
    sim = gpu_run(G, gates, n, d, 81, 1e-12)
    ref = oracle_run(gates, n, d, 81, 1e-12)
    assert max(ref.mps.bond_dims()) >= 9 or max(sim.stats()["max_chi"], 0) >= 9
    assert sim.decisions() == ref.decisions
    st = sim.stats()
    assert st["vn_evaluations"] < st["candidates_scored"]
    err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
    assert err < TOL


def _planted_theta(kind, d, cl, cr, seed):
    """theta (chi_l, d, d, chi_r) whose matrix M (chi_l d x d chi_r) has row 0 = e_0, so the first
    Gram column below the diagonal, (M M^H)[1:, 0], is M[1:, 0] exactly and becomes the first
    Householder vector of the tridiagonalisation.  'subnormal': a complex subnormal pivot (its
    phase x0 / |x0| is of modulus 1 only if x0 is rescaled first) over a random tail; 'tail': a
    pivot 1 over a tail 1e-8 that |x|^2 - |x0|^2 would cancel to zero."""
    rng = np.random.default_rng(seed)
    rows, cols = cl * d, d * cr
    M = (rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))) / np.sqrt(2 * cols)
    M[0] = 0
    M[0, 0] = 1.0
    if kind == "subnormal":
        M[1, 0] = complex(3e-321, 4e-321)
    else:
        M[1, 0], M[2, 0], M[3:, 0] = 1.0, 1e-8, 0.0
    return M.reshape(cl, d, d, cr)


def _renyi2(theta, u):
    cl, d, _, cr = theta.shape
    tq = np.einsum("uv,avb->aub", u, theta.reshape(cl, d * d, cr)).reshape(cl * d, d * cr)
    p = np.linalg.svd(tq, compute_uv=False) ** 2
    p = p / p.sum()
    return -np.log(np.sum(p * p))


@pytest.mark.parametrize("kind,cl,cr,seed,tol", [("subnormal", 3, 3, 7, TOL), ("subnormal", 9, 27, 7, TOL),
                                                 ("tail", 3, 3, 5, 1e-12)])
def test_score_theta_householder_edge_cases(G, kind, cl, cr, seed, tol):
    """Scores of every class for a planted theta against the oracle's SVD entropies.  The identity
    class sees the planted Gram column; with the plain phase quotient its entropy is off by ~1e-5
    (subnormal), with the cancelled tail by ~1e-9 (tail), while FP64 rounding of the exact
    method stays below 1e-14.  Both warp-level (9 x 9) and CTA-level (27 x 81) scoring are
    covered; score_theta evaluates every class exactly, the disentangler's own choice (returned
    with it) goes through the Renyi-2 pruning."""
    d = 3
    theta = _planted_theta(kind, d, cl, cr, seed)
    ref = GCAMPS(8, d, chi_max=81)
    want = ref.score_bond(theta)
    sim = G.Simulator(8, d, chi_max=81)
    s2, vn, choice, nev = sim.score_theta(theta)
    assert abs(vn[0] - want[0]) < tol
    assert np.max(np.abs(vn - want)) < tol
    assert choice == ref.choose(want)
    assert 1 <= nev <= len(want)   # the Renyi-2 bound prunes at every size
    r2 = np.array([_renyi2(theta, u) for (_s, _i, u) in ref.cands])
    assert np.max(np.abs(s2 - r2)) < TOL


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("d,n,layers,t,seed,chi", [(3, 8, 10, 14, 41, 81), (2, 10, 10, 10, 3, 64),
                                                   (3, 12, 12, 16, 31, 64)])
def test_score_kinds_match_oracle(G, kind, d, n, layers, t, seed, chi):
    """Renyi-2 (kind 1) and weight-rank (kind 2) scores: decisions and bond dimensions equal the
    oracle's (which scores every class by SVD), and the state stays exact."""
    gates = brickwork_circuit(n, d, layers, t, seed)
    sim = G.Simulator(n, d, chi_max=chi, cutoff=1e-12, score_kind=kind)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    ref = GCAMPS(n, d, chi_max=chi, cutoff=1e-12, score_kind=kind)
    for gt in gates:
        ref.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            ref.disentangle()
    assert sim.decisions() == ref.decisions
    assert sim.bond_dims() == ref.mps.bond_dims()
    assert any(k for _b, k in ref.decisions)
    if d ** n <= 6561:
        err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
        assert err < TOL
    sim.close()


def test_uneven_batch_matches_oracle_per_circuit(G):
    """One handle with circuits of different qudit counts (the batched form): each circuit's
    tableau, decisions, bond dimensions and state equal the oracle's run of that circuit alone, and
    a smaller cluster size set after creation gives the same results."""
    d = 3
    ns = [5, 8, 6, 7, 4]
    gates = [brickwork_circuit(n, d, n, n, 100 + n) for n in ns]
    ops, begin = [], [0]
    for n, g in zip(ns, gates):
        o = G.ops_from_gates(g, d)
        ops.append(o)
        begin.append(begin[-1] + len(o))
    sim = G.Simulator(ns, d, chi_max=81, cutoff=1e-12, cluster_size=4)
    assert sim.batch == len(ns) and [sim._lib.gcamps_num_qudits(sim._h, c) for c in range(len(ns))] == ns
    for csize in (4, 2):
        sim.set_cluster_size(csize)
        sim.reset()
        sim.run(np.concatenate(ops), begin)
        sim.sync()
        for c, (n, g) in enumerate(zip(ns, gates)):
            ref = oracle_run(g, n, d, 81, 1e-12)
            e, p = sim.tableau(c)
            re_, rp = ref.tab.exps_phase()
            assert np.array_equal(e, re_) and np.array_equal(p, rp)
            assert sim.decisions(c) == ref.decisions
            assert sim.bond_dims(c) == ref.mps.bond_dims()
            err, _ = sv.same_up_to_phase(sim.statevector(c), sv.run(g, n, d))
            assert err < TOL
    with pytest.raises(G.GcampsError):
        sim.set_cluster_size(8)          # above the size the scratch was laid out for
    sim.close()


@pytest.mark.parametrize("scale", [1e-9, 1e9])
def test_score_theta_of_badly_scaled_tensors(G, scale):
    """Entropies do not depend on the scale of theta; far from unit norm the FP32 screen gives no
    bound and every class is evaluated exactly, so scores and choice still equal the oracle's."""
    d, cl, cr = 3, 9, 9
    rng = np.random.default_rng(21)
    shape = (cl * d, d * cr)
    r = 4
    m = (rng.standard_normal((shape[0], r)) + 1j * rng.standard_normal((shape[0], r))) @ \
        (rng.standard_normal((r, shape[1])) + 1j * rng.standard_normal((r, shape[1])))
    theta = (m / np.linalg.norm(m) * scale).reshape(cl, d, d, cr)
    ref = GCAMPS(8, d, chi_max=81)
    want = ref.score_bond(theta)
    sim = G.Simulator(8, d, chi_max=81)
    s2, vn, choice, nev = sim.score_theta(theta)
    assert np.max(np.abs(vn - want)) < TOL
    assert choice == ref.choose(want)
    sim.close()


@pytest.mark.parametrize("d", [2, 3])
def test_two_qudit_circuits(G, d):
    """The smallest system (n = 2, one bond): T gates and disentangling against the dense state."""
    n = 2
    for seed in (1, 2, 3):
        gates = brickwork_circuit(n, d, 4, 4, seed)
        sim = gpu_run(G, gates, n, d, 9, 1e-14)
        ref = oracle_run(gates, n, d, 9, 1e-14)
        assert sim.decisions() == ref.decisions
        assert sim.bond_dims() == ref.mps.bond_dims()
        err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
        assert err < TOL
        sim.close()


def test_chi_max_one_truncates_to_a_product_state(G):
    """chi_max = 1: every truncation keeps one Schmidt value; both sides keep the same product state
    and discard the same weight."""
    d, n = 3, 5
    gates = brickwork_circuit(n, d, 5, 5, 11)
    sim = gpu_run(G, gates, n, d, 1, 1e-12)
    ref = oracle_run(gates, n, d, 1, 1e-12)
    assert sim.bond_dims() == ref.mps.bond_dims() == [1] * (n - 1)
    assert sim.decisions() == ref.decisions
    assert abs(sim.stats()["discarded_weight"] - ref.discarded) < 1e-10
    err, _ = sv.same_up_to_phase(sim.statevector(), ref.statevector())
    assert err < 1e-9
    sim.close()


def test_empty_gate_list_leaves_the_initial_state(G):
    d, n = 3, 4
    sim = G.Simulator(n, d, chi_max=9)
    sim.run(np.zeros(0, dtype=G.OP_DTYPE))
    sim.sync()
    e, p = sim.tableau()
    ref = oracle_run([], n, d, 9, 1e-12)
    re_, rp = ref.tab.exps_phase()
    assert np.array_equal(e, re_) and np.array_equal(p, rp)
    assert sim.bond_dims() == [1] * (n - 1) and sim.decisions() == []
    psi = sim.statevector()
    assert abs(abs(psi[0]) - 1.0) < 1e-14 and np.sum(np.abs(psi[1:])) < 1e-14
    sim.close()


def test_largest_qudit_count_clifford_tableau(G):
    """n = 128 (the largest supported): a Clifford-only brickwork gives the oracle's tableau bit for bit,
    and a T gate then reads its Weyl string from the inverse tableau."""
    d, n = 2, 128
    gates = [g for g in brickwork_circuit(n, d, 6, 1, 3) if hasattr(g, "sp_index")]
    sim = G.Simulator(n, d, chi_max=4, cutoff=1e-12)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    ref = clifford_oracle_tableau(gates, n, d)
    e, p = sim.tableau()
    assert np.array_equal(e, ref[0]) and np.array_equal(p, ref[1])
    sim.close()


def clifford_oracle_tableau(gates, n, d):
    g = GCAMPS(n, d, chi_max=4, cutoff=1e-12)
    for gt in gates:
        g.apply_gate(gt)
    return g.tab.exps_phase()


@pytest.mark.parametrize("d", [2, 3])
def test_named_gates_match_oracle(G, d):
    """gcamps_apply_named (H, S, SUM in either qudit order, X, Z) against the oracle's dense conjugation
    of the same matrices: forward and inverse tableaux bit for bit."""
    from oracle.weyl import X, Z
    n = 4
    sim = G.Simulator(n, d, chi_max=8)
    ref = GCAMPS(n, d, chi_max=8)
    one = {G.GATE_H: clifford.H_gate(d), G.GATE_S: clifford.S_gate(d), G.GATE_X: X(d), G.GATE_Z: Z(d)}
    rng = np.random.default_rng(60 + d)
    for _step in range(40):
        gate = int(rng.integers(1, 6))
        if gate == G.GATE_SUM:
            q0, q1 = (int(v) for v in rng.choice(n, 2, replace=False))
            sim.apply_named(gate, q0, q1)
            ref.apply_clifford([q0, q1], clifford.images_by_conjugation(clifford.SUM_gate(d), 2, d))
        else:
            q = int(rng.integers(n))
            sim.apply_named(gate, q)
            ref.apply_clifford([q], clifford.images_by_conjugation(one[gate], 1, d))
    sim.sync()
    assert_same_tableaux(sim, ref)
    with pytest.raises(G.GcampsError):
        sim.apply_named(G.GATE_SUM, 0)
    with pytest.raises(G.GcampsError):
        sim.apply_named(G.GATE_H, 0, 1)
    sim.close()


@pytest.mark.parametrize("d,n,layers", [(3, 6, 12), (2, 8, 16)])
def test_layer_by_layer_runs_match_oracle(G, d, n, layers):
    """The circuit family of Fig. 4 (a random Clifford on all qudits, then a T gate on qudit 0, per
    layer), run one layer per launch on one handle as the bond-dimension-per-layer experiment does:
    the bond dimensions after every layer and all decisions equal the oracle's, and the final state is
    exact (chi_max = d^floor(n/2) never binds).  The seeded circuits cover both regimes of Fig. 5a: a
    product-state MPS for about n layers, then growth."""
    from synth import layered_t_circuit
    gates, ends = layered_t_circuit(n, d, layers, 1)
    chi = d ** (n // 2)
    sim = G.Simulator(n, d, chi_max=chi, cutoff=1e-12)
    ref = GCAMPS(n, d, chi_max=chi, cutoff=1e-12)
    a = 0
    seen = []
    for b in ends:
        sim.run(G.ops_from_gates(gates[a:b], d))
        for gt in gates[a:b]:
            ref.apply_gate(gt)
            if not hasattr(gt, "sp_index"):
                ref.disentangle()
        dims = sim.bond_dims()
        assert dims == ref.mps.bond_dims(), b
        seen.append(max(dims))
        a = b
    sim.sync()
    assert seen[0] == 1 and max(seen) > d
    assert sim.decisions() == ref.decisions
    err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
    assert err < TOL
    sim.close()


def _spectrum_theta(kind, d, cl, cr, seed):
    """theta whose matrix (chi_l d x d chi_r) has a planted Schmidt spectrum, between random isometries:
    'flat' rank 3 with equal weights (a 3-fold degenerate eigenvalue and zeros), 'decay' weights 2^-k
    down to 2^-(m-1) (many small eigenvalues inside one FP32 bracket), 'pairs' eigenvalues in pairs
    split by one part in 1e9, 'zeros' rank 2 (the rest of the Gram's eigenvalues are rounding noise)."""
    rng = np.random.default_rng(seed)
    rows, cols = cl * d, d * cr
    m = min(rows, cols)
    if kind == "flat":
        w = np.zeros(m)
        w[:3] = 1.0
    elif kind == "decay":
        w = 2.0 ** -np.arange(m)
    elif kind == "pairs":
        base = 1.5 ** -np.arange((m + 1) // 2)
        w = np.repeat(base, 2)[:m] * np.tile([1.0, 1.0 + 1e-9], (m + 1) // 2)[:m]
    else:
        w = np.zeros(m)
        w[:2] = [0.7, 0.3]
    qa, _ = np.linalg.qr(rng.standard_normal((rows, m)) + 1j * rng.standard_normal((rows, m)))
    qb, _ = np.linalg.qr(rng.standard_normal((cols, m)) + 1j * rng.standard_normal((cols, m)))
    M = (qa * np.sqrt(w / w.sum())) @ qb.conj().T
    return M.reshape(cl, d, d, cr)


@pytest.mark.parametrize("kind", ["flat", "decay", "pairs", "zeros"])
@pytest.mark.parametrize("cl,cr", [(3, 3), (9, 9), (27, 27)])
def test_score_theta_spectra_that_stress_the_eigenvalue_refinement(G, kind, cl, cr):
    """Every class's von Neumann entropy for thetas whose spectra exercise the FP64 refinement of the
    FP32 eigenvalue brackets (Newton steps kept only where Sturm counts verify them, multisection
    otherwise) at warp-level (m = 9), CTA-level short-list (m = 27) and CTA-level (m = 81) sizes, against
    the oracle's SVD entropies at 1e-10; the chosen class is the oracle's."""
    d = 3
    theta = _spectrum_theta(kind, d, cl, cr, 100 + cl + cr)
    ref = GCAMPS(8, d, chi_max=81)
    want = ref.score_bond(theta)
    sim = G.Simulator(8, d, chi_max=81)
    s2, vn, choice, nev = sim.score_theta(theta)
    assert np.max(np.abs(vn - want)) < TOL, (kind, cl, float(np.max(np.abs(vn - want))))
    assert choice == ref.choose(want)
