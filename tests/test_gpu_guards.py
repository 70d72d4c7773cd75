"""Writes past the ends of device buffers, checked with guard bands (opt.guard_bands = 1)
in place of a memory checker: every buffer of a handle lies between two 4096-byte bands
of a fill byte, and after the work of every form on a ragged lattice (V/2 not a multiple
of the block size, every extent different, odd t-slices) no band has changed."""
import numpy as np
import pytest
import torch

from paper_1010_4782_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1010_4782_gb300 import build

    build.build()
    binding.load()


FORMS = [
    dict(arith=binding.STAG_ARITH_F64),
    dict(arith=binding.STAG_ARITH_FF),
    dict(arith=binding.STAG_ARITH_FF, long_recon=12, long_scale=inputs.NAIK_COEFF),
    dict(arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_F32),
    dict(arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_F32, long_recon=12, long_scale=inputs.NAIK_COEFF),
    dict(arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_F16),
    dict(arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_BF16),
    dict(arith=binding.STAG_ARITH_FF, inner=binding.STAG_INNER_F32_L16),
    dict(arith=binding.STAG_ARITH_F64, timing=1, use_graphs=0),
]


@pytest.mark.parametrize("form", range(len(FORMS)))
def test_guard_bands_intact_after_every_call(form):
    dims, mass = (10, 6, 4, 12), 0.05
    fat, lng = inputs.asqtad_form_fields(dims, seeds=(91, 92, 93))
    opt = binding.stag_default_options()
    opt.guard_bands = 1
    for k, v in FORMS[form].items():
        setattr(opt, k, v)
    with binding.Handle(torch.from_numpy(fat).cuda(), dims, mass, naik_long=torch.from_numpy(lng).cuda(),
                        options=opt) as h:
        vh = int(np.prod(dims)) // 2
        v = torch.from_numpy(inputs.gaussian_even_source(dims, 94)).cuda()
        out = torch.empty_like(v)
        binding.stag_apply_A(h.h, v, out)
        for p_out in (0, 1):
            binding.stag_dslash(h.h, p_out, v, out)
        x = torch.zeros_like(v)
        code, info = binding.stag_cg_solve(h.h, v, x, 1e-10, max_iter=20000)
        assert code == binding.STAG_OK, info
        checked, bad = binding.stag_check_guards(h.h)
    assert checked >= 2 * 4096 * 10 and bad == 0, (checked, bad)
    assert vh % 256 != 0


def test_guard_check_needs_guard_bands():
    dims = (4, 4, 4, 4)
    with binding.Handle(torch.from_numpy(inputs.gauge_field(dims, 1)).cuda(), dims, 0.1) as h:
        with pytest.raises(binding.StagError):
            binding.stag_check_guards(h.h)
