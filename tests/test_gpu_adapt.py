"""Adaptation decisions on the GPU (Sec. 4.1, 4.3, 4.4): smoothness sensor, adjoint-weighted
element indicator, Doerfler marking and the h/p choice, against the oracle."""
import numpy as np
import pytest

import oracle as O
from hdg_testlib import lib_params, oracle_params, rel_err
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1308_3995_gb300 import hdg
    return hdg.Context(0)


def _mark_gpu(ctx, eta2, sensor, theta, eps_s):
    from paper_1308_3995_gb300 import hdg
    e = torch.from_numpy(np.ascontiguousarray(eta2, dtype=np.float64)).to("cuda:0")
    s = torch.from_numpy(np.ascontiguousarray(sensor, dtype=np.float64)).to("cuda:0")
    code = torch.full((e.numel(),), -1, dtype=torch.int8, device="cuda:0")
    nm = hdg.adapt_mark(ctx, e, s, code, theta=theta, eps_s=eps_s)
    torch.cuda.synchronize()
    return code.cpu().numpy(), nm


@pytest.mark.parametrize("n,kind", [(1, "rand"), (4, "hand"), (7, "ties"), (1000, "rand"), (1000, "ties"),
                                    (1000, "zeros"), (262144, "rand"), (262144, "heavy")])
@pytest.mark.parametrize("theta", [0.05, 0.5, 0.0])
def test_marking_bit_exact_against_oracle(ctx, n, kind, theta):
    rng = np.random.default_rng(n + int(100 * theta))
    if kind == "hand":
        eta2 = np.array([1.0, 4.0, 9.0, 16.0])
    elif kind == "ties":
        eta2 = rng.integers(0, 4, size=n).astype(np.float64)     # many exact ties and zeros
    elif kind == "zeros":
        eta2 = np.zeros(n); eta2[rng.integers(0, n, 5)] = 1.0
    elif kind == "heavy":
        eta2 = rng.pareto(1.2, size=n) ** 2                     # a few elements carry most of the error
    else:
        eta2 = rng.exponential(size=n) ** 3
    sensor = 10.0 ** rng.uniform(-9, -3, size=n)
    sensor[np.abs(np.log10(sensor) + 6) < 1e-9] = 1e-3          # nothing on the threshold itself
    code_o, nm_o = O.adapt_mark(eta2, sensor, theta=theta, eps_s=1e-6)
    code_g, nm_g = _mark_gpu(ctx, eta2, sensor, theta, 1e-6)
    assert nm_g == nm_o and np.array_equal(code_g, code_o)


@pytest.mark.parametrize("name,nx,ny,kw", [("euler_p3_16k", 6, 7, {}), ("ns_mixp_65k", 5, 6, {}),
                                           ("ns_mixp_65k", 6, 6, {"model": 0})])
def test_indicators_against_oracle(ctx, name, nx, ny, kw):
    """S_K against the oracle's quadrature form; eta_K^2 = (res_u,K . U~_K)^2 against the oracle's
    residual with the same adjoint coefficients."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS[name], nx, ny, **kw)
    case = G.make_case(wl)
    om = O.Mesh(case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, _ = G.case_state(case, om.face_vid, om.face_p)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    sysm = hdg.System(ctx, mesh, lib_params(wl))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    Ua = np.random.default_rng(9).standard_normal(mesh.u_len)
    Uat = torch.from_numpy(Ua).to(dev)
    sysm.condense(Ut, Lt)
    eta2 = torch.empty(mesh.n_elem, dtype=torch.float64, device=dev)
    sens = torch.empty_like(eta2)
    sysm.adapt_indicators(Ut, Uat, eta2, sens)
    torch.cuda.synchronize()
    s_ref = np.array([om.smoothness(K, U) for K in range(om.n_elem)])
    assert rel_err(sens.cpu().numpy(), s_ref) < 1e-13
    ru = om.condense(oracle_params(wl), U, Lam)["res_u"]
    eg = eta2.cpu().numpy()
    for K in range(om.n_elem):
        sl = slice(om.u_off[K], om.u_off[K + 1])
        d = float(ru[sl] @ Ua[sl])
        scale = float(np.abs(ru[sl]) @ np.abs(Ua[sl]))
        assert abs(np.sqrt(eg[K]) - abs(d)) < 1e-12 * scale + 1e-300
    sysm.close(); mesh.close()


def test_adaptation_pipeline_primal_adjoint_mark(ctx):
    """Newton step state -> adjoint (Sec. 4.2) -> indicators -> Doerfler + h/p on the GPU; the codes
    equal the oracle's marking of the same indicator arrays, and the marked share holds."""
    from paper_1308_3995_gb300 import hdg
    wl = G.small_variant(G.WORKLOADS["euler_p3_262k_shock"], 24, 32)
    case = G.make_case(wl)
    mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
    U, Lam, _ = G.case_state(case, mesh.face_vid, mesh.face_p)
    cfl = 10.0
    primal = hdg.System(ctx, mesh, lib_params(wl, cfl))
    adj = hdg.System(ctx, mesh, lib_params(wl, cfl))
    dev = torch.device("cuda:0")
    Ut, Lt = torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)
    Ft = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    nb = 10                                   # J = integral of density: F~ on the density constant mode
    Ft.view(-1, 4 * nb)[:, 0] = 1.0
    primal.condense(Ut, Lt)
    adj.adjoint_condense(primal, Ut, Lt, Ft)
    solver = hdg.Solver(primal, restart=40)
    lt = torch.zeros(mesh.lam_len, dtype=torch.float64, device=dev)
    ua = torch.zeros(mesh.u_len, dtype=torch.float64, device=dev)
    solver.solve(lt, rtol=1e-10, max_iter=2000, rhs=adj.views()["E"], transpose=True)
    adj.recover(lt, ua)
    eta2 = torch.empty(mesh.n_elem, dtype=torch.float64, device=dev)
    sens = torch.empty_like(eta2)
    primal.adapt_indicators(Ut, ua, eta2, sens)
    code = torch.empty(mesh.n_elem, dtype=torch.int8, device=dev)
    nm = hdg.adapt_mark(ctx, eta2, sens, code, theta=0.05, eps_s=1e-6)
    torch.cuda.synchronize()
    e, s, c = eta2.cpu().numpy(), sens.cpu().numpy(), code.cpu().numpy()
    code_o, nm_o = O.adapt_mark(e, s, theta=0.05, eps_s=1e-6)
    assert nm == nm_o and np.array_equal(c, code_o)
    assert e[c > 0].sum() >= 0.95 ** 2 * e.sum() * (1 - 1e-12)
    print("marked", nm, "of", mesh.n_elem, "p-enrichment", int((c == 1).sum()), "h-refinement", int((c == 2).sum()))
    solver.close(); adj.close(); primal.close(); mesh.close()
