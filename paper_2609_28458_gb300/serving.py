"""The mixed serving batch: three independent ensembles that one GPU serves at once (the paper's
three applications, Secs. 3-5), issued as one CUDA graph by ``api.MixedBatch``.

* profile-likelihood fits (Sec. 4.3): n_lam slopes x n_mock mock data sets, 20 Gauss-Newton
  iterations each, every iteration a flatness solve with its forward sensitivities (graph-safe,
  FP64: with FP32 stages chi^2 is too noisy for the fits' convergence test);
* Milky-Way orbits (Sec. 3 setting): forward solve recording the step tape, then the discrete
  adjoint of the endpoint loss 1/2 |y(t1) - y_tgt|^2 with respect to y0 and the potential;
* binary spin precession (Sec. 5): Verner 7 in FP64, forward recording the tape, then the adjoint of
  the summed cosines of the final spin tilts, cos theta_j = S_j . L, with respect to y0 and (q, chi1, chi2).

Each piece owns its workspaces; ``pieces(...)`` returns callables(sm_limit) for ``api.MixedBatch``
and ``autotune.share_sms``.
"""
import numpy as np
import torch

from . import api
from . import workloads as W


def pieces(n_lam=100, n_mock=100, n_mw=1 << 18, n_prec=1 << 17, mw_precision="fp32df", device="cuda"):
    dev = torch.device(device)
    out = {}

    # profile-likelihood fits
    data = W.profile_data(n_lam=n_lam)
    bao, sn = W.profile_truth_lcdm(data)
    C_bao = W.bao_covariance(data, bao)
    pd = api.ProfileData(data.z_nodes, data.bao_z, data.bao_kind, np.linalg.cholesky(C_bao), data.z_sn,
                         np.linalg.cholesky(data.sn_cov), W.profile_mocks(bao, C_bao, n_mock, seed=5002),
                         W.profile_mocks(sn, data.sn_cov, n_mock, seed=5003), device=dev)
    lam = torch.as_tensor(np.repeat(data.lam_grid, n_mock), device=dev)
    mock = torch.as_tensor(np.tile(np.arange(n_mock), n_lam), dtype=torch.int32, device=dev)
    ws_fit = api.Workspace(dev)

    def fits(sm):
        return api.profile_fit(pd, lam, mock, workspace=ws_fit, n_iter=20, graph_safe=1, sm_limit=sm,
                               precision="fp64", rtol=1e-8, atol=1e-11, gtol=1e-10)

    out["fits"] = fits

    # Milky-Way orbit gradients
    e = W.mw(n=n_mw, seed=1000)
    rtol_mw = 1e-8
    y0 = torch.as_tensor(e.y0, device=dev)
    pr = torch.as_tensor(e.params, device=dev)
    t0, t1, sv = (torch.as_tensor(x, device=dev) for x in (e.t0, e.t1, e.saveat))
    ptgt = pr.clone()
    ptgt[:, :3] *= 1.01
    y_tgt = api.solve("mw", y0, ptgt, t0, t1, sv, rtol_mw, rtol_mw, precision="fp64")["y"].clone()
    probe = api.solve("mw", y0, pr, t0, t1, sv, rtol_mw, rtol_mw, precision=mw_precision)
    nb_mw = int(api.tape_bytes("mw", n_mw, n_accept=(probe["n_accept"].double() * 1.2).ceil().int(),
                               precision=mw_precision))
    ws_mw = api.Workspace(dev)

    def orbits(sm):
        s = api.solve("mw", y0, pr, t0, t1, sv, rtol_mw, rtol_mw, precision=mw_precision, kernel="persistent",
                      record_tape=True, workspace=ws_mw, tape_nbytes=nb_mw, sm_limit=sm)
        g = api.vjp("mw", y0, pr, t0, t1, sv, rtol_mw, rtol_mw, s["y"] - y_tgt, precision=mw_precision,
                    kernel="persistent", reuse_tape=s, workspace=ws_mw, sm_limit=sm)
        return dict(y=s["y"], status=s["status"], dLdy0=g["dLdy0"], dLdparams=g["dLdparams"])

    out["orbits"] = orbits

    # precession gradients
    p = W.precession(n=n_prec, seed=2000)
    rtol_p = 3.16e-9
    py0 = torch.as_tensor(p.y0, device=dev)
    pp = torch.as_tensor(p.params, device=dev)
    pt0, pt1, psv = (torch.as_tensor(x, device=dev) for x in (p.t0, p.t1, p.saveat))
    probe = api.solve("precession", py0, pp, pt0, pt1, psv, rtol_p, rtol_p, method="vern7", precision="fp64")
    nb_p = int(api.tape_bytes("precession", n_prec, n_accept=(probe["n_accept"].double() * 1.2).ceil().int(),
                              precision="fp64"))
    ws_p = api.Workspace(dev)

    def precession(sm):
        s = api.solve("precession", py0, pp, pt0, pt1, psv, rtol_p, rtol_p, method="vern7", precision="fp64",
                      kernel="persistent", record_tape=True, workspace=ws_p, tape_nbytes=nb_p, sm_limit=sm)
        y = s["y"][:, -1]
        w = torch.cat([y[:, 3:6] + y[:, 6:9], y[:, 0:3], y[:, 0:3]], dim=1).unsqueeze(1)
        g = api.vjp("precession", py0, pp, pt0, pt1, psv, rtol_p, rtol_p, w, method="vern7", precision="fp64",
                    kernel="persistent", reuse_tape=s, workspace=ws_p, sm_limit=sm)
        return dict(y=s["y"], status=s["status"], dLdy0=g["dLdy0"], dLdparams=g["dLdparams"])

    out["precession"] = precession
    return out
