"""The CG error bounds of the paper (Prop. 1, classical; Prop. 3, with sigma_0 the eigenvalues
outside a cluster; Sec. 4) against the GPU's own FP64 CG iterates on the random-vector
workload of Example 1b (m = p, H = I, N = 50, Q = 0.1 I, R = I): the energy-norm error of the
iterate after r steps (enkf fixed_iters = r, the solution Z read back through
enkf_copy_intermediates) lies below both bounds wherever they are above the round-off floor,
equals the oracle's CG error, and at m = 1000, where the spectrum is a cluster at 1 with
N - 1 outliers, Prop. 3 predicts the step count far better than Prop. 1."""
import numpy as np
import pytest

import oracle
from oracle import blockcg as bc
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("m", [200, 1000])
def test_gpu_cg_errors_against_prop1_and_prop3(lib, m):
    p = synth.ex1b_problem(m)
    N = p.N
    _, _, Z, _, HA = oracle.ensemble_stats(p.Xf, p.rowptr, p.col, p.w)
    D = oracle.innovations(p.y, Z, None)
    S = HA @ HA.T / (N - 1) + np.diag(p.r)
    eigs = np.linalg.eigvalsh(S)
    Zs = np.linalg.solve(S, D)
    e0 = float(np.mean(np.sqrt(np.einsum("ij,ij->j", Zs, S @ Zs))))
    _, info = oracle.cgd_enkf(p.Xf, p.rowptr, p.col, p.w, p.r, p.y, None, fixed_iters=25, keep_iterates=True)
    ref_err = bc.energy_errors(S, D, info["iterates"])
    Xf = torch.from_numpy(p.Xf).cuda()
    y = torch.from_numpy(p.y).cuda()
    steps_needed = {}
    for r in (1, 2, 5, 10, 15, 20, 25):
        an = lib.Analysis(m, m, N, p.rowptr, p.col, p.w, p.r, precision="fp64", fixed_iters=r, perturb_obs=0)
        an.analyze(Xf, y)
        _, _, Zg, _ = an.intermediates()
        E = Zs - Zg.cpu().numpy()
        err = float(np.mean(np.sqrt(np.einsum("ij,ij->j", E, S @ E))))
        cl = bc.classical_bound(eigs, r) * e0
        p3 = bc.prop3_best(eigs, r, max_out=8) * e0
        floor = 1e-9 * e0
        if cl > floor:
            assert err <= cl * (1 + 1e-9), (m, r, err, cl)
        if p3 > floor:
            assert err <= p3 * (1 + 1e-9), (m, r, err, p3)
        assert abs(err - ref_err[r]) <= 1e-6 * ref_err[r] + 1e-12 * e0, (r, err, ref_err[r])
        steps_needed[r] = (err, cl, p3)
        an.close()
    if m == 1000:
        err10, cl10, p310 = steps_needed[10]
        assert p310 < 1e-2 * cl10 and err10 <= p310
