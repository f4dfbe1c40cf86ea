"""Multi-shot inversion iteration (ews_fwi_iteration): batched gradients of
several shots on one model, their sum, a scaled steepest-descent step with a
parabolic step length.  Pinned by: the summed gradient direction equals the
sum of single-shot gradients (checked through the first trial model), and
the misfit decreases monotonically over iterations towards a model that
explains the data (a +10 % sphere hidden in a layered background)."""
import numpy as np
import pytest

from paper_2112_15071_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ews():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_15071_gb300 import ews as E
    E.load()
    return E


def setting(ews):
    import torch
    base = synth.small_problem(44, 40, 36, nt=140, boundary="sponge", width=6, kind="moment",
                               nrec=12, seed=4)
    true_vp, true_vs, true_rho = synth.add_sphere(base.vp, base.vs, base.spacing,
                                                  [22 * base.spacing[0], 20 * base.spacing[1],
                                                   18 * base.spacing[2]], 60.0, 0.10)
    srcs = [np.array([x, y, 9 * base.spacing[2]]) for x, y in
            ((12.3 * base.spacing[0], 11.1 * base.spacing[1]),
             (31.4 * base.spacing[0], 12.7 * base.spacing[1]),
             (20.6 * base.spacing[0], 29.2 * base.spacing[1]))]
    shots = []
    for s in srcs:
        sim_t = ews.Simulation(base.nx, base.ny, base.nz, base.spacing, boundary="sponge",
                               width=base.width)
        sim_t.set_model_vel(true_vp, true_vs, true_rho)
        sim_t.set_source("moment", s, base.src_comp, base.wavelet)
        sim_t.set_receivers(base.rec_pos)
        obs = torch.from_numpy(sim_t.run(base.nt, base.dt)).cuda()
        sim_t.close()
        sim = ews.Simulation(base.nx, base.ny, base.nz, base.spacing, boundary="sponge",
                             width=base.width)
        sim.set_model_vel(base.vp, base.vs, base.rho)
        sim.set_source("moment", s, base.src_comp, base.wavelet)
        sim.set_receivers(base.rec_pos)
        shots.append({"sim": sim, "nt": base.nt, "dt": base.dt, "observed": obs})
    lam, mu, rho = (torch.from_numpy(a).cuda() for a in base.lame())
    return base, shots, lam, mu, rho


def test_misfit_decreases_over_iterations(ews):
    base, shots, lam, mu, rho = setting(ews)
    J = []
    for it in range(4):
        j0, j1, a = ews.ews_fwi_iteration(shots, lam, mu, rho, max_rel_step=0.02, ckpt_every=40)
        if J:
            assert j0 == pytest.approx(J[-1], rel=1e-5)       # same model, same misfit
        else:
            J.append(j0)
        J.append(j1)
        assert a > 0 and j1 < j0, (it, j0, j1, a)
    print("misfits:", J)
    assert J[-1] < 0.92 * J[0]          # measured: 0.88 after 4 iterations


def test_summed_gradient_is_the_sum_of_shot_gradients(ews):
    """The first trial model equals m - a s_p sum_s g_s computed from
    single-shot gradients (ews_gradient) on the host."""
    import torch
    base, shots, lam, mu, rho = setting(ews)
    m0 = [t.cpu().numpy().astype(np.float64) for t in (lam, mu, rho)]
    gsum = [np.zeros_like(m0[0]) for _ in range(3)]
    for d in shots:
        mis, g = d["sim"].gradient(d["nt"], d["dt"], d["observed"].cpu().numpy(), ckpt_every=40)
        for q in range(3):
            gsum[q] += g[q]
    j0, j1, a = ews.ews_fwi_iteration(shots, lam, mu, rho, max_rel_step=0.01, ckpt_every=40)
    assert a > 0
    got = [t.cpu().numpy().astype(np.float64) for t in (lam, mu, rho)]
    for q in range(3):
        sc = np.abs(m0[q]).max() / np.abs(gsum[q]).max()
        want = m0[q] - a * sc * gsum[q]
        inside = np.abs(a * sc * gsum[q]) < 0.4 * np.abs(m0[q])          # clamps inactive
        err = np.abs(got[q] - want)[inside].max() / np.abs(m0[q]).max()
        assert err <= 1e-5, (q, err)
