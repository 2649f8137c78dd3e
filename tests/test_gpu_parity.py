"""CUDA path vs the complex128 oracle, element by element, through the C ABI.

Tolerances: symbolic analysis bit-exact; complex128 operators, fronts and preconditioner
applications within 1e-10 relative (Frobenius / 2-norm); GMRES solutions at a true relative
residual below 1e-5 measured by the oracle's own sparse matvec on the host.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import discretize as dz
from oracle import gmres as ogm
from oracle import panels as opn
from oracle import symbolic as osy
from oracle import sweep as osw
from paper_1204_0111_gb300 import workloads as wl

from _cases import Case, small_cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1204_0111_gb300 import psp  # noqa: E402

CASES = small_cases()
IDS = [c.name for c in CASES]
_oracles = {}


def oracle_for(case: Case, mode="moving"):
    key = (case.name, mode)
    if key not in _oracles:
        _oracles[key] = osw.SweepingPreconditioner(case.oracle_problem(), case.depth, case.pad, case.leaf, mode=mode)
    return _oracles[key]


def gpu_for(case: Case, precision="c128", mode="moving", **kw):
    c = torch.from_numpy(case.c).cuda()
    return psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                      pml_C=case.C, alpha=case.alpha, precision=precision, faces=case.faces, mode=mode,
                                      **kw)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_symbolic_bit_exact(case):
    P = gpu_for(case)
    plan = opn.panel_plan(case.nz, case.gamma, case.depth)
    assert P.info()["panels"] == len(plan)
    for i, (z0, z1) in enumerate(plan):
        meta, sns = psp.parse_symbolic(P.symbolic(i))
        lead = 0 if z0 == 0 else case.pad
        assert (meta["nx"], meta["ny"], meta["nz"], meta["lead"]) == (case.nx, case.ny, lead + z1 - z0, lead)
        ref = osy.nested_dissection(case.nx, case.ny, lead + z1 - z0, case.leaf)
        assert meta["nsn"] == len(ref.supernodes)
        for (s, u, par, nodes, struct), sn in zip(sns, ref.supernodes):
            assert s == len(sn.nodes) and u == len(sn.struct) and par == sn.parent
            assert np.array_equal(nodes, sn.nodes) and np.array_equal(struct, sn.struct)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_matvec_A_and_J(case):
    P = gpu_for(case)
    p = case.oracle_problem()
    x = wl.random_vector(case.N, 3, seed=11)
    xd = torch.from_numpy(x).cuda()
    for which, M in ((0, dz.operator_A(p)), (1, dz.operator_J(p))):
        yd = torch.empty_like(xd)
        P.matvec(xd, yd, which)
        ref = (M @ x.T).T
        assert rel(yd.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_front_factors(case):
    P = gpu_for(case)
    O = oracle_for(case)
    worst = 0.0
    for i in range(O.m):
        for f, fr in enumerate(O.fronts[i]):
            G, s, u = P.export_front(i, f)
            Linv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
            top = np.tril(Linv, -1) + np.diag(fr.d)
            exp = np.vstack([top, fr.L_BL @ Linv])
            got = G.copy()
            got[:s] = np.tril(got[:s])
            worst = max(worst, rel(got, exp))
    assert worst < 1e-10, worst


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("nrhs", [1, 3])
def test_apply_matches_oracle(case, nrhs):
    P = gpu_for(case)
    O = oracle_for(case)
    r = wl.random_vector(case.N, nrhs, seed=21 + nrhs)
    ref = O.apply(r)
    rd = torch.from_numpy(r).cuda()
    out = torch.empty_like(rd)
    P.apply(rd, out)
    assert rel(out.cpu().numpy(), ref) < 1e-10
    # in place, and through host buffers
    P.apply(rd, rd)
    assert rel(rd.cpu().numpy(), ref) < 1e-10
    host_out = np.zeros_like(r)
    P.apply(r, host_out)
    assert rel(host_out, ref) < 1e-10


@pytest.mark.parametrize("si", ["extended", "paper", "two"])
@pytest.mark.parametrize("max_rows", [128, 256])
def test_whole_front_up_tasks_match_oracle(max_rows, si):
    # up-the-tree tasks of up to 128 or 256 rows (a whole front per task at the bottom of the tree);
    # one task per level is enough (sweep_level_tasks 1), so the small case's levels keep the full
    # width instead of halving it towards the 8-row floor
    case = CASES[2]
    c = torch.from_numpy(case.c).cuda()
    P = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                   pml_C=case.C, alpha=case.alpha, faces=case.faces, sweep_max_rows=max_rows,
                                   sweep_level_tasks=1, selective_inversion=si)
    r = wl.random_vector(case.N, 3, seed=33)
    out = np.zeros_like(r)
    P.apply(r, out)
    assert rel(out, oracle_for(case).apply(r)) < 1e-10
    P.close()


def test_exact_mode_is_inverse_of_J():
    case = CASES[1]
    P = gpu_for(case, mode="exact")
    p = case.oracle_problem()
    x = wl.random_vector(case.N, 2, seed=5)
    Jx = (dz.operator_J(p) @ x.T).T
    out = np.zeros_like(x)
    P.apply(np.ascontiguousarray(Jx), out)
    assert rel(out, x) < 1e-9


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_gmres_solve_converges_like_oracle(case):
    P = gpu_for(case)
    O = oracle_for(case)
    p = case.oracle_problem()
    A = dz.operator_A(p)
    f = wl.gaussian_source(case.nx, case.ny, case.nz, case.h, (0.5, 0.5, 0.5))
    b = dz.rhs_scale(p) * f
    _, it_oracle, _ = ogm.gmres(lambda v: A @ v, O.apply, b, tol=1e-5, k=20, maxit=300)
    fd = torch.from_numpy(f[None, :].copy()).cuda()
    ud = torch.zeros_like(fd)
    info = P.solve(fd, ud, tol=1e-5, k=20, maxit=300)
    u = ud.cpu().numpy()[0]
    true_rel = np.linalg.norm(b - A @ u) / np.linalg.norm(b)
    assert info["converged"] == 1 and true_rel < 1e-5
    assert abs(info["iterations"] - it_oracle) <= 1


def test_gmres_several_shots_and_nonconvergence():
    case = CASES[0]
    P = gpu_for(case)
    p = case.oracle_problem()
    A = dz.operator_A(p)
    srcs = [(0.5, 0.5, 0.5), (0.3, 0.6, 0.2), (0.7, 0.2, 0.8)]
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, s) for s in srcs])
    fd = torch.from_numpy(f).cuda()
    ud = torch.zeros_like(fd)
    info = P.solve(fd, ud, tol=1e-6, k=10, maxit=300)
    u = ud.cpu().numpy()
    b = dz.rhs_scale(p)[None, :] * f
    for j in range(3):
        assert np.linalg.norm(b[j] - A @ u[j]) / np.linalg.norm(b[j]) < 1e-6
    assert info["restarts"] >= 1
    with pytest.raises(psp.PSPError) as e:
        P.solve(fd, ud, tol=1e-6, k=10, maxit=2)
    assert e.value.name == "PSP_ERR_NOT_CONVERGED"


@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_complex64_path_solves_to_tolerance(case):
    P64 = gpu_for(case, precision="c64")
    O = oracle_for(case)
    r = wl.random_vector(case.N, 1, seed=3)
    ref = O.apply(r)
    out = np.zeros_like(r)
    P64.apply(r, out)
    err = rel(out, ref)
    assert err < 1e-3          # single-precision fronts: the apply differs at ~1e-6..1e-4
    p = case.oracle_problem()
    A = dz.operator_A(p)
    f = wl.gaussian_source(case.nx, case.ny, case.nz, case.h, (0.5, 0.5, 0.5))[None, :].copy()
    u = np.zeros_like(f)
    info = P64.solve(f, u, tol=1e-5, k=20, maxit=300)
    b = dz.rhs_scale(p) * f[0]
    assert np.linalg.norm(b - A @ u[0]) / np.linalg.norm(b) < 1e-5 and info["converged"] == 1


@pytest.mark.parametrize("case", CASES[1:], ids=IDS[1:])
def test_complex64_diagonal_blocks_in_fp64(case):
    # complex64 factors whose diagonal blocks (their LDL^T and the solves against them) are computed in
    # complex128: every stored front and the application stay within complex64 accuracy of the
    # oracle, and on the fronts without children (whose inputs both paths round alike) the pivots of
    # the first diagonal block agree with the oracle's more closely, on average, than the
    # all-complex64 factorisation's do
    c = torch.from_numpy(case.c).cuda()
    kw = dict(pad=case.pad, leaf=case.leaf, pml_C=case.C, alpha=case.alpha, precision="c64", faces=case.faces)
    Pw = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, diag_fp64=True, **kw)
    Pn = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, **kw)
    O = oracle_for(case)
    worst, dw, dn = 0.0, [], []
    for i in range(O.m):
        sns = O.sym[i].supernodes
        for f, fr in enumerate(O.fronts[i]):
            Gw, s, u = Pw.export_front(i, f)
            Gn, _, _ = Pn.export_front(i, f)
            Linv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
            exp = np.vstack([np.tril(Linv, -1) + np.diag(fr.d), fr.L_BL @ Linv])
            got = Gw.copy()
            got[:s] = np.tril(got[:s])
            worst = max(worst, rel(got, exp))
            if not sns[f].children:
                b = min(s, 32)
                dw.append(rel(np.diag(Gw[:b, :b]), fr.d[:b]))
                dn.append(rel(np.diag(Gn[:b, :b]), fr.d[:b]))
    assert worst < 1e-3, worst
    assert dw and np.mean(dw) < np.mean(dn), (np.mean(dw), np.mean(dn))
    r = wl.random_vector(case.N, 1, seed=5)
    out = np.zeros_like(r)
    Pw.apply(r, out)
    assert rel(out, O.apply(r)) < 1e-3
    Pw.close()
    Pn.close()


def test_single_panel_and_zero_pivot_free_small_grid():
    # panel depth >= nz: one auxiliary problem, M^{-1} = J^{-1}
    case = Case(np.ones((7, 5, 6)), 1.0 / 8, 5.0, 1, 50, leaf=8)
    P = gpu_for(case)
    assert P.info()["panels"] == 1
    p = case.oracle_problem()
    J = dz.operator_J(p).toarray()
    x = wl.random_vector(case.N, 1, seed=9)
    out = np.zeros_like(x)
    P.apply(np.ascontiguousarray((J @ x.T).T), out)
    assert rel(out, x) < 1e-10


@pytest.mark.parametrize("case", CASES[1:], ids=IDS[1:])
def test_tensor_core_fronts_complex64(case):
    # complex64 fronts with the long contractions on tcgen05 (split-TF32, 3 real products) against
    # the same path on CUDA cores and against the complex128 oracle
    c = torch.from_numpy(case.c).cuda()
    kw = dict(pad=case.pad, leaf=case.leaf, pml_C=case.C, alpha=case.alpha, precision="c64", faces=case.faces)
    Ptc = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, tensor_cores=True, **kw)
    Pcc = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, tensor_cores=False, **kw)
    O = oracle_for(case)
    worst_tc, worst_cc, worst_diff = 0.0, 0.0, 0.0
    big = False   # fronts with s, u >= 96 take the 128 x 128 tensor-core tiles
    for i in range(O.m):
        for f, fr in enumerate(O.fronts[i]):
            Gt, s, u = Ptc.export_front(i, f)
            Gc, _, _ = Pcc.export_front(i, f)
            big = big or (s >= 96 and u >= 96)
            if u == 0:
                continue
            Linv = sla.solve_triangular(fr.L_TL, np.eye(s), lower=True, unit_diagonal=True)
            exp = fr.L_BL @ Linv
            worst_tc = max(worst_tc, rel(Gt[s:], exp))
            worst_cc = max(worst_cc, rel(Gc[s:], exp))
            worst_diff = max(worst_diff, rel(Gt[s:], Gc[s:]))
    assert worst_cc < 1e-3 and worst_tc < 1e-3 and worst_diff < 1e-3, (worst_tc, worst_cc, worst_diff)
    st = Ptc.stats()
    assert (st.get("k_tc_gemm", {}).get("launches", 0) > 0) == big


@pytest.mark.parametrize("precision", ["c128", "c64"])
@pytest.mark.parametrize("si", ["extended", "paper"])
def test_claiming_one_task_ahead_gives_the_same_bits(si, precision):
    # a sweep CTA holding one queue task besides the one it runs, instead of two, changes which CTA
    # runs what and when, not the arithmetic: the same bits, for one and for several right-hand sides
    case = CASES[2]
    for nrhs in (1, 3):
        r = wl.random_vector(case.N, nrhs, seed=45)
        outs = []
        for ca in (2, 1):
            P = gpu_for(case, selective_inversion=si, precision=precision, sweep_claim_ahead=ca)
            out = np.zeros_like(r)
            P.apply(r, out)
            P.close()
            outs.append(out)
        assert np.array_equal(outs[0], outs[1])
        assert rel(outs[1], oracle_for(case).apply(r)) < (1e-10 if precision == "c128" else 1e-4)


def test_sweep_autotuner_keeps_results():
    case = CASES[2]
    P = gpu_for(case)
    O = oracle_for(case)
    t = P.tune_sweep(nrhs=2, reps=1)
    assert t["sweep_level_tasks"] in (152, 304, 608, 1216, 2432)
    assert t["sweep_ctas_per_sm"] in (2, 3, 4, 6, 8) and t["sweep_rhs_group"] in (0, 1, 2)
    assert t["sweep_max_rows"] in (64, 128, 256) and t["sweep_claim_ahead"] in (1, 2)
    assert t["candidates"] >= 10 and 0 < t["best_ms"] <= t["initial_ms"]
    r = wl.random_vector(case.N, 2, seed=44)
    out = np.zeros_like(r)
    P.apply(r, out)
    assert rel(out, O.apply(r)) < 1e-10


def test_solve_in_groups_of_right_hand_sides_equals_one_run():
    # psp_solve may split the right-hand sides into several GMRES runs (when their bases do not fit
    # in memory together); every column iterates independently, so the solutions are the same
    case = CASES[0]
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, s)
                  for s in ((0.5, 0.5, 0.5), (0.3, 0.6, 0.2), (0.7, 0.2, 0.8))])
    P = gpu_for(case)
    u1 = np.zeros_like(f)
    i1 = P.solve(f, u1, tol=1e-6, k=10, maxit=300)
    c = torch.from_numpy(case.c).cuda()
    Q = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                   pml_C=case.C, alpha=case.alpha, faces=case.faces, solve_rhs_group=1)
    u3 = np.zeros_like(f)
    i3 = Q.solve(f, u3, tol=1e-6, k=10, maxit=300)
    assert i1["groups"] == 1 and i3["groups"] == 3
    assert np.array_equal(u1, u3)
    assert i3["iterations"] == i1["iterations"] and i3["converged"] == 1


def test_runs_of_right_hand_sides_are_balanced():
    # seven columns with room for three per run: three runs (3, 2, 2), the same solutions as one run
    # (to rounding: a sweep over 8, 4 or 2 columns stages its vectors in chunks of different lengths,
    # which changes the order of the column sums down the tree)
    case = CASES[0]
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, (0.2 + 0.1 * j, 0.5, 0.3 + 0.05 * j))
                  for j in range(7)])
    c = torch.from_numpy(case.c).cuda()
    kw = dict(pad=case.pad, leaf=case.leaf, pml_C=case.C, alpha=case.alpha, faces=case.faces)
    P = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, **kw)
    Q = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, solve_rhs_group=3, **kw)
    u1, u3 = np.zeros_like(f), np.zeros_like(f)
    i1 = P.solve(f, u1, tol=1e-6, k=10, maxit=300)
    i3 = Q.solve(f, u3, tol=1e-6, k=10, maxit=300)
    assert i1["groups"] == 1 and i3["groups"] == 3
    assert i3["iterations"] == i1["iterations"] and i3["converged"] == 1
    assert np.linalg.norm(u3 - u1) / np.linalg.norm(u1) < 1e-10
    P.close()
    Q.close()


def test_gmres_v_only_basis_matches_z_basis():
    # right preconditioning: x0 + M^{-1}(V y) equals x0 + Z y with z_j = M^{-1} v_j; keeping V only costs
    # one more application per restart cycle (k = 6 forces several cycles)
    case = CASES[1]
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, s) for s in ((0.5, 0.5, 0.5), (0.3, 0.6, 0.2))])
    out = {}
    for basis in ("z", "v"):
        c = torch.from_numpy(case.c).cuda()
        P = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                       pml_C=case.C, alpha=case.alpha, faces=case.faces, gmres_basis=basis)
        u = np.zeros_like(f)
        out[basis] = (P.solve(f, u, tol=1e-8, k=6, maxit=300), u)
        P.close()
    (iz, uz), (iv, uv) = out["z"], out["v"]
    assert iz["converged"] == 1 and iv["converged"] == 1
    assert iv["iterations"] == iz["iterations"] and iv["restarts"] == iz["restarts"] and iz["restarts"] > 1
    assert iv["applies"] == iz["applies"] + iv["restarts"]
    assert np.linalg.norm(uv - uz) / np.linalg.norm(uz) < 1e-9


def test_allocator_callbacks_own_every_device_allocation():
    # the caller's allocator (here torch's caching allocator) receives every allocation of the handle;
    # results are those of a handle using cudaMalloc, and a failing allocator gives PSP_ERR_OOM
    case = CASES[2]
    live, calls = {}, [0]

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        calls[0] += 1
        return p

    def free(p):
        torch.cuda.caching_allocator_delete(p)
        del live[p]

    c = torch.from_numpy(case.c).cuda()
    kw = dict(pad=case.pad, leaf=case.leaf, pml_C=case.C, alpha=case.alpha, faces=case.faces)
    P = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, allocator=(alloc, free), **kw)
    Q = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, **kw)
    assert sum(live.values()) >= P.info()["factor_bytes"] > 0
    x = torch.from_numpy(wl.random_vector(case.N, 2, seed=4)).cuda()
    a, b = torch.empty_like(x), torch.empty_like(x)
    P.apply(x, a)
    Q.apply(x, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    f = wl.gaussian_source(case.nx, case.ny, case.nz, case.h, (0.5, 0.5, 0.5))[None, :].copy()
    u = np.zeros_like(f)
    assert P.solve(f, u, tol=1e-6, k=10, maxit=200)["converged"] == 1
    n_before = calls[0]
    P.close()
    Q.close()
    assert not live and calls[0] == n_before
    with pytest.raises(psp.PSPError) as e:
        psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, allocator=(lambda n: 0, free), **kw)
    assert e.value.name == "PSP_ERR_OOM"


def test_solve_history_and_pivot_monitor():
    case = CASES[1]
    O = oracle_for(case)
    dmin = min(float(np.min(np.abs(fr.d))) for fronts in O.fronts.values() for fr in fronts)
    P = gpu_for(case)
    f = np.stack([wl.gaussian_source(case.nx, case.ny, case.nz, case.h, s) for s in ((0.5, 0.5, 0.5), (0.2, 0.7, 0.3))])
    u = np.zeros_like(f)
    info = P.solve(f, u, tol=1e-8, k=5, maxit=300)
    assert abs(info["min_pivot_abs"] - dmin) <= 1e-12 * dmin
    est, true = P.solve_history(0), P.solve_history(1)
    assert est.shape == (info["iterations"], 2) and true.shape == (info["restarts"], 2)
    assert np.all(est[-1] < 1e-8) and np.all(est > 0)
    assert np.max(true[-1]) == pytest.approx(info["relres_max"], rel=1e-12)
    # within a restart cycle the GMRES residual estimate does not increase
    for c0 in range(0, info["iterations"], 5):
        cyc = est[c0:c0 + 5]
        assert np.all(np.diff(cyc, axis=0) <= 1e-12 * cyc[:-1])
    P.close()


def test_sweep_wait_gives_up_and_the_device_stays_usable():
    # a dependency of the persistent sweep that can never be met (test option): its bounded wait
    # gives up after about two seconds, psp_solve reports PSP_ERR_TIMEOUT, and a normal handle
    # solves afterwards on the same device
    case = CASES[0]
    c = torch.from_numpy(case.c).cuda()
    f = wl.gaussian_source(case.nx, case.ny, case.nz, case.h, (0.5, 0.5, 0.5))[None, :].copy()
    P = psp.SweepingPreconditioner(c, case.h, case.omega, case.gamma, case.depth, pad=case.pad, leaf=case.leaf,
                                   pml_C=case.C, alpha=case.alpha, faces=case.faces, test_sweep_stall=1)
    u = np.zeros_like(f)
    with pytest.raises(psp.PSPError) as e:
        P.solve(f, u, tol=1e-6, k=10, maxit=50)
    assert e.value.name == "PSP_ERR_TIMEOUT"
    P.check_status()                       # psp_solve reported the give-up and cleared the flag
    # psp_apply with a host output synchronises and reports the give-up itself
    with pytest.raises(psp.PSPError) as e:
        P.apply(f, np.zeros_like(f))
    assert e.value.name == "PSP_ERR_TIMEOUT"
    # with device pointers it only enqueues; psp_check_status reports it once
    fd = torch.from_numpy(f).cuda()
    P.apply(fd, torch.empty_like(fd))
    with pytest.raises(psp.PSPError) as e:
        P.check_status()
    assert e.value.name == "PSP_ERR_TIMEOUT"
    P.check_status()
    P.close()
    Q = gpu_for(case)
    u = np.zeros_like(f)
    assert Q.solve(f, u, tol=1e-6, k=10, maxit=300)["converged"] == 1
