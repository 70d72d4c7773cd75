"""Parity of the further forms at their workload sizes, checked on sampled sites
with the oracle's single-site A (Sec. 2, Eq. (3)); the whole-lattice oracle is
too slow here.  Each solve must meet |b - A x| / |b| <= 10 tol on the sample
(the library's own FP64 check covers the whole lattice):

  * mixed FP32 reliable-update CG on the 28^3 x 96 asqtad-form system, with
    nine-entry and with two-row Naik links;
  * the batch of 16 right-hand sides on 32^3 x 64 (asqtad-form) together with
    uneven one-hop lattices (8^4, 16^4, 24^3 x 48), in one batched solve;
  * flexible CG with the network at its polynomial start on 32^3 x 64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

N_SAMPLES = 32
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


def _sampled_rel_residual(fat, lng, mass, dims, b, x, seed):
    vh = int(np.prod(dims)) // 2
    rng = np.random.default_rng(seed)
    sites = np.concatenate([[0, vh - 1], rng.choice(vh, N_SAMPLES - 2, replace=False)])
    num = den = 0.0
    for i in sites:
        s = oracle.even_site_coords(dims, int(i))
        r = b[i] - oracle.apply_A_at(fat, lng, mass, x, s, dims)
        num += np.vdot(r, r).real
        den += np.vdot(b[i], b[i]).real
    return np.sqrt(num / den)


@pytest.mark.parametrize("long_recon", [0, 12])
def test_mixed_fp32_at_28x28x28x96(long_recon):
    """Mixed FP32 at the workload size, with nine-entry Naik links and with two-row
    Naik links (long_recon = 12, third row rebuilt in FP32 and in float-float)."""
    dims, mass = (28, 28, 28, 96), 0.0062
    fat, lng = inputs.asqtad_form_fields(dims)
    b = inputs.gaussian_even_source(dims, 0)
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_FF
    opt.inner = binding.STAG_INNER_F32
    if long_recon:
        opt.long_recon, opt.long_scale = 12, inputs.NAIK_COEFF
    with binding.Handle(torch.from_numpy(fat).cuda(), dims, mass, naik_long=torch.from_numpy(lng).cuda(),
                        options=opt) as h:
        x = torch.zeros_like(torch.from_numpy(b).cuda())
        code, info = binding.stag_cg_solve(h.h, torch.from_numpy(b).cuda(), x, TOL, max_iter=40000)
    assert code == binding.STAG_OK and info["true_rel_residual"] <= TOL, info
    assert info["reliable_updates"] >= 1 and info["fallbacks"] == 0
    assert _sampled_rel_residual(fat, lng, mass, dims, b, x.cpu().numpy(), 7) <= 10 * TOL


def test_batch_16_rhs_at_32x32x32x64_with_uneven_lattices():
    main = (32, 32, 32, 64)
    fat, lng = inputs.asqtad_form_fields(main, seeds=(21, 22, 23))
    fat_d, lng_d = torch.from_numpy(fat).cuda(), torch.from_numpy(lng).cuda()
    systems = [(fat, lng, fat_d, lng_d, main, 0.0062, inputs.gaussian_even_source(main, k)) for k in range(16)]
    for j, (d, m) in enumerate([((8, 8, 8, 8), 0.01), ((16, 16, 16, 16), 0.03), ((24, 24, 24, 48), 0.05)]):
        f = inputs.gauge_field(d, 500 + j)
        systems.append((f, None, torch.from_numpy(f).cuda(), None, d, m, inputs.gaussian_even_source(d, 600 + j)))
    bt = binding.stag_batch_create([s[2] for s in systems], [s[3] for s in systems], [s[4] for s in systems],
                                   [s[5] for s in systems])
    try:
        bs = [torch.from_numpy(s[6]).cuda() for s in systems]
        xs = [torch.zeros_like(b) for b in bs]
        code, infos = binding.stag_batch_solve(bt, bs, xs, TOL, 40000)
    finally:
        binding.stag_batch_destroy(bt)
    assert code == binding.STAG_OK, infos
    assert all(i["true_rel_residual"] <= TOL for i in infos)
    # right-hand sides 0 and 15 of the multi-RHS group, and the three uneven lattices
    for k in (0, 15, 16, 17, 18):
        f, l, _, _, d, m, b = systems[k]
        assert _sampled_rel_residual(f, l, m, d, b, xs[k].cpu().numpy(), 11 + k) <= 10 * TOL, k


def test_fcg_polynomial_start_at_32x32x32x64():
    dims, mass = (32, 32, 32, 64), 0.0062
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(31, 32, 33))
    b = inputs.gaussian_even_source(dims, 90000)
    opt = binding.stag_default_options()
    opt.arith = binding.STAG_ARITH_FF
    with binding.Handle(torch.from_numpy(fat).cuda(), dims, mass, naik_long=torch.from_numpy(lng).cuda(),
                        options=opt) as h:
        net = binding.stag_ptnet_create(h.h, binding.STAG_ARITH_BF16, 5)
        try:
            x = torch.zeros_like(torch.from_numpy(b).cuda())
            code, info = binding.stag_fcg_solve(h.h, net, torch.from_numpy(b).cuda(), x, TOL, 40000)
        finally:
            binding.stag_ptnet_destroy(net)
    assert code == binding.STAG_OK and info["true_rel_residual"] <= TOL, info
    assert info["fallbacks"] == 0
    assert _sampled_rel_residual(fat, lng, mass, dims, b, x.cpu().numpy(), 13) <= 10 * TOL
