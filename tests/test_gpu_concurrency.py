"""Systems of different meshes condensed at once from several host threads,
each on its own stream, give bitwise the results each gives alone.  The
degree buckets of these mixed-degree meshes are launched in groups of trace
sizes, each launch with shared memory for its own largest trace; the
kernels' dynamic shared-memory cap is one value per kernel instance shared
by all threads (the instance's largest layout), so no thread can lower it
under another thread's launch."""
import threading

import pytest

from hdg_testlib import lib_params
from paper_1308_3995_gb300 import inputs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_REPEAT = 20


def _systems(ctx, precision):
    from paper_1308_3995_gb300 import hdg
    mix = (0.4, 0.3, 0.2, 0.1)
    wls = [G.small_variant(G.WORKLOADS["ns_mixp_65k"], 6 + 2 * i, 12 + 4 * i, seed=100 + i) for i in range(4)]
    wls += [G.small_variant(G.WORKLOADS["euler_p3_16k"], 8 + 2 * i, 16 + 4 * i, p=None, probs=mix, seed=200 + i)
            for i in range(4)]
    dev = torch.device("cuda:0")
    out = []
    for wl in wls:
        case = G.make_case(wl)
        mesh = hdg.Mesh(ctx, case.mesh.elem_xy, case.mesh.elem_vid, case.elem_p, case.nfield, case.mesh.elem_bc)
        sysm = hdg.System(ctx, mesh, lib_params(wl, 0.0, precision))
        U, Lam, _ = G.case_state(case, mesh.face_vid, mesh.face_p)
        out.append((mesh, sysm, torch.from_numpy(U).to(dev), torch.from_numpy(Lam).to(dev)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_threads_condensing_mixed_meshes_at_once_match_alone(precision):
    from paper_1308_3995_gb300 import hdg
    ctx = hdg.Context(0)
    items = _systems(ctx, precision)
    alone = []
    for _, sysm, U, Lam in items:
        sysm.condense(U, Lam)
        torch.cuda.synchronize()
        assert sysm.launches >= 1
        alone.append({k: t.clone() for k, t in sysm.views().items()})
    errors = []

    def work(i):
        try:
            _, sysm, U, Lam = items[i]
            st = torch.cuda.Stream()
            for _ in range(N_REPEAT):
                sysm.condense(U, Lam, stream=st)
            st.synchronize()
        except Exception as exc:  # reported by the main thread
            errors.append((i, repr(exc)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(items))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    torch.cuda.synchronize()
    for i, (_, sysm, _, _) in enumerate(items):
        got = sysm.views()
        for k, ref in alone[i].items():
            assert torch.equal(got[k], ref), f"system {i}: {k} differs after concurrent condensation"
