"""The library's ab initio environment (Eq. 1 from integrals) on the host.

A host-only context builds the operator-table and block operators (the
renormalisation runs as host loops there); the test applies H_eff from the
library's own task table and operator blocks with NumPy and compares it with
the oracle (a different operator-table, the same H_eff), with full CI when
the bonds keep every multiplet, and compares the renormalised block
Hamiltonians block by block.
"""
import numpy as np
import pytest

import synth
from oracle import abinitio, fci, heff, sectors

L_ = pytest.importorskip("paper_2309_16724_gb300._lib")


def lib_apply(env, sec):
    rows, v = env.tasks()
    A_op, D_op, _, _ = env.terms()
    blocks, n = sec.blocks, sec.psi_len
    cache = {}

    def op(side, oid, qo, qi):
        key = (side, oid, qo, qi)
        if key not in cache:
            S = sec.left if side == 0 else sec.right
            cache[key] = env.operator_block(side, oid, qo, qi, S[qo][2], S[qi][2])
        return cache[key]

    def apply(psi):
        F = np.zeros(n)
        for (f, term, e, ao, ai, bo, bi, flags), vv in zip(rows, v):
            B, Fb = blocks[e], blocks[f]
            X = psi[B[8]:B[8] + B[6] * B[7]].reshape(B[7], B[6]).T
            if not flags & 2:
                X = X @ op(1, D_op[term], bo, bi).T
            if not flags & 1:
                X = op(0, A_op[term], ao, ai) @ X
            F[Fb[8]:Fb[8] + Fb[6] * Fb[7]] += vv * X.T.reshape(-1)
        return F
    return apply


@pytest.fixture(scope="module")
def hctx():
    import paper_2309_16724_gb300 as P
    return P.Context(-1)


def build_both(hctx, cfg):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    sec, env = workload.build(hctx, cfg, model=P.SU2_MODEL_AB_INITIO)
    table, oenv, lsec, rsec = abinitio.build_problem(cfg)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    tasks = heff.build_tasks(table, left, right, blocks, cfg.twoS)
    return sec, env, lambda psi: heff.apply_heff(table, oenv, tasks, blocks, n, psi), oenv, lsec, rsec


@pytest.mark.parametrize("L,N,twoS,D", [(6, 5, 1, 400), (7, 8, 2, 400), (10, 9, 1, 40), (12, 12, 0, 60)])
def test_library_environment_matches_oracle(hctx, L, N, twoS, D):
    cfg = synth.Config("ab", synth.SPATIAL_ORBITAL, L, N, twoS, D, 1002)
    sec, env, oapply, oenv, lsec, rsec = build_both(hctx, cfg)
    apply = lib_apply(env, sec)
    for seed in (1, 2):
        psi = synth.gaussian_psi(sec.psi_len, seed)
        F, G = apply(psi), oapply(psi)
        assert np.linalg.norm(F - G) <= 1e-13 * np.linalg.norm(G)
    # the renormalised block Hamiltonians (left / right operator 1) block by block
    for side, name, S in ((0, "L", lsec), (1, "R", rsec)):
        for (qo, qi), M in oenv[(name, 1)].items():
            Mb = env.operator_block(side, 1, qo, qi, S[qo][2], S[qi][2])
            assert np.abs(Mb - M).max() <= 1e-12 * max(1.0, np.abs(M).max())


def test_library_heff_spectrum_equals_full_ci(hctx):
    cfg = synth.Config("ab", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    sec, env = workload.build(hctx, cfg, model=P.SU2_MODEL_AB_INITIO)
    apply = lib_apply(env, sec)
    n = sec.psi_len
    Hm = np.array([apply(np.eye(n)[i]) for i in range(n)]).T
    ev = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))
    h, eri = synth.integrals(6, 1002)
    ref = fci.spin_levels(h, eri, 6, 0)
    assert len(ev) == len(ref)
    assert np.abs(ev - ref).max() < 1e-11
    assert env.info["renorm_flops"] > 0


def test_ab_initio_argument_errors(hctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("ab", synth.SPATIAL_ORBITAL, 6, 6, 0, 20, 1002)
    with pytest.raises(P.Su2Error) as ei:       # integrals missing
        lch, rch = workload.chains(cfg)
        sec = P.Sectors(hctx, lch[-1], rch[-1], cfg.site_kind, cfg.N, cfg.twoS)
        P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch, rch, n_left=cfg.n_left, n_right=cfg.n_right)
    assert ei.value.code == P._lib.SU2_EINVAL
    h, eri = synth.integrals(6, 1002)
    with pytest.raises(P.Su2Error) as ei:       # integral shapes
        P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch, rch, n_left=cfg.n_left, n_right=cfg.n_right,
                      h=h[:5, :5], eri=eri)
    assert ei.value.code == P._lib.SU2_EINVAL
    with pytest.raises(P.Su2Error) as ei:       # a chain shorter than the block
        P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch[1:], rch, n_left=cfg.n_left, n_right=cfg.n_right,
                      h=h, eri=eri)
    assert ei.value.code == P._lib.SU2_EINVAL


@pytest.mark.parametrize("n_left", [0, 1, 2, 3, 4])
def test_every_bond_position_equals_full_ci(hctx, n_left):
    """The window at every position of an L = 6 chain, empty blocks at the
    ends included: with bonds that keep every multiplet, the lowest
    eigenvalue of the library's H_eff (built densely from its task table and
    operator blocks) is the full-CI ground-state energy."""
    import paper_2309_16724_gb300 as P
    L, N = 6, 6
    cfg = synth.Config("ab", synth.SPATIAL_ORBITAL, L, N, 0, 400, 1002)
    h, eri = synth.integrals(L, 1002)
    nr = L - 2 - n_left
    lch, rch = synth.bond_sector_chain(cfg, n_left), synth.bond_sector_chain(cfg, nr)
    sec = P.Sectors(hctx, lch[-1], rch[-1], cfg.site_kind, N, 0)
    env = P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch, rch, n_left=n_left, n_right=nr, seed=1002, h=h, eri=eri)
    apply = lib_apply(env, sec)
    n = sec.psi_len
    H = np.stack([apply(np.eye(n)[i]) for i in range(n)], 1)
    assert np.abs(H - H.T).max() <= 1e-13
    assert abs(np.linalg.eigvalsh(H)[0] - fci.spin_levels(h, eri, N, 0)[0]) <= 1e-12
    env.close()


def random_tensors(chain, rng):
    """Random orthonormal MPS tensors along a bond chain: per step the
    oracle's {sector: (stacked rows, Q)} and the flat array in the layout of
    su2_hamiltonian's mps_left / mps_right."""
    from oracle import sweep as osweep
    sites = synth.site_states(synth.SPATIAL_ORBITAL)
    steps, flat = [], []
    for k in range(1, len(chain)):
        A = {}
        for qo, (Nq, Sq, d) in enumerate(chain[k]):
            rows, r0 = osweep._stacks(chain[k - 1], sites, Nq, Sq)
            Q, _ = np.linalg.qr(rng.standard_normal((r0, d)))
            A[qo] = (rows, Q)
            flat.append(Q.ravel(order="F"))
        steps.append(A)
    return steps, np.concatenate(flat)


@pytest.mark.parametrize("L,N,twoS,D", [(8, 8, 0, 30), (9, 7, 1, 24)])
def test_caller_mps_tensors_match_oracle(hctx, L, N, twoS, D):
    """An environment built from the caller's MPS tensors (random orthonormal
    Q per step, both blocks) equals the oracle's blocks grown with the same
    tensors: H.psi through the library's task table and operator blocks
    against the oracle's H_eff."""
    import paper_2309_16724_gb300 as P
    cfg = synth.Config("ab", synth.SPATIAL_ORBITAL, L, N, twoS, D, 1002)
    h, eri = synth.integrals(L, 1002)
    rng = np.random.default_rng(5)
    lch, rch = synth.bond_sector_chain(cfg, cfg.n_left), synth.bond_sector_chain(cfg, cfg.n_right)
    lsteps, lflat = random_tensors(lch, rng)
    rsteps, rflat = random_tensors(rch, rng)
    sec = P.Sectors(hctx, lch[-1], rch[-1], cfg.site_kind, N, twoS)
    env = P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch, rch, n_left=cfg.n_left, n_right=cfg.n_right,
                        seed=1002, h=h, eri=eri, mps_left=lflat, mps_right=rflat)
    strings = abinitio.hamiltonian_strings(h, eri)
    Lb, Rb = abinitio.LeftBlock(strings, L), abinitio.RightBlock(strings, L)
    for k, A in enumerate(lsteps, start=1):
        Lb = Lb.grown(lch[k], A)
    for k, A in enumerate(rsteps, start=1):
        Rb = Rb.grown(rch[k], A)
    table, oenv, ls, rs = abinitio.problem_from_blocks(strings, Lb, Rb)
    blocks, n = sectors.build_blocks(ls, rs, cfg.site_kind, N, twoS)
    assert n == sec.psi_len
    tasks = heff.build_tasks(table, ls, rs, blocks, twoS)
    apply = lib_apply(env, sec)
    for seed in (1, 2):
        psi = synth.gaussian_psi(n, seed)
        F = heff.apply_heff(table, oenv, tasks, blocks, n, psi)
        G = apply(psi)
        assert np.linalg.norm(G - F) <= 1e-13 * np.linalg.norm(F)
    # the seeded tensors differ from these: the caller's tensors were used
    env0 = P.Environment(hctx, sec, P.SU2_MODEL_AB_INITIO, lch, rch, n_left=cfg.n_left, n_right=cfg.n_right,
                         seed=1002, h=h, eri=eri)
    psi = synth.gaussian_psi(n, 3)
    assert np.linalg.norm(lib_apply(env0, sec)(psi) - apply(psi)) > 1e-6 * np.linalg.norm(apply(psi))
    env.close()
    env0.close()
