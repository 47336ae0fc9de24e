"""axpic_step_noalloc, the entry point for callers that cannot allocate device
memory (their memory manager owns the GPU heap, or an allocation could stall a
real-time loop), against axpic_step on the same plasma: two steps in a row,
through the C ABI. Collected last so that a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300 import AxionPlasma, _lib  # noqa: E402

FIELDS = ("w", "px", "py", "pz", "x", "y", "z")


def _plasmas(ncells, prm):
    n = 6e25 / 1.1
    n_ion = np.tile([[0.9 * n, 0.1 * n]], (ncells, 1))
    T = np.linspace(1.5, 4.5, ncells)
    args = (ncells, T, n_ion, [1.0, 2.0], [1.00794, 4.002602], 1e-12, (64, 192, 512), prm)
    ref = AxionPlasma(*args[:-1], dict(prm, diag_enable=1))
    ref.sample(61, 37, 13)
    other = AxionPlasma(*args)   # owns a second copy of the slabs; its context is not used to step
    other.sample(61, 37, 13)
    torch.cuda.synchronize()
    return ref, other


def test_noalloc_step_matches_context_step_twice():
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3e9, seed=77, T_mode=2, relax_r=0.2,
               tally_enable=0, diag_enable=0)
    ncells = 40
    ref, other = _plasmas(ncells, prm)
    carry = torch.zeros(4 * ncells, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for step in (0, 1):
        res_before = ref.residuals()
        ref.step(step, _lib.CH_ALL)
        _lib.axpic_step_noalloc(other.desc, other.params, step, _lib.CH_ALL, carry.data_ptr(), stream)
        torch.cuda.synchronize()
        for c in range(ncells):
            a, b = ref.cell(c), other.cell(c)
            for k in "ega":
                assert len(a[k]["w"]) == len(b[k]["w"]), (step, c, k)
                for f in FIELDS:
                    np.testing.assert_allclose(b[k][f], a[k][f], rtol=1e-5, atol=1e-6 * np.abs(a[k][f]).max(initial=0),
                                               err_msg="step %d cell %d %s.%s" % (step, c, k, f))
        np.testing.assert_allclose(other.temperatures(), ref.temperatures(), rtol=1e-5)
        # the carried exchange is what binary32 momenta could not take; the two
        # paths sum the electron moments in different orders, so it agrees to
        # a small fraction of the exchange each cell requested
        res_ref = ref.residuals()
        res_na = carry.reshape(ncells, 4).cpu().numpy()
        dg = ref.cell_diag()
        reqE = np.abs(dg[:, 0] + res_before[:, 0])
        reqP = np.linalg.norm(dg[:, 1:4] + res_before[:, 1:4], axis=1)
        assert np.all(np.abs(res_na[:, 0] - res_ref[:, 0]) <= 1e-3 * reqE + 1e-6), step
        assert np.all(np.linalg.norm(res_na[:, 1:] - res_ref[:, 1:], axis=1) <= 1e-3 * reqP + 1e-9), step
    ref.close()
    other.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    prm = dict(g_agg_GeV_inv=1e-10, g_ae=1e-12, dt_phys_s=2e12, w_a=3e9)
    ref, other = _plasmas(4, prm)
    desc = _lib.PlasmaDesc.from_buffer_copy(other.desc)
    desc.ncells = 16385
    carry = torch.zeros(4 * 4, dtype=torch.float64, device="cuda")
    st = _lib.lib().axpic_step_noalloc(desc, other.params, 0, 7, carry.data_ptr(), None)
    assert st == _lib.AXPIC_E_INVALID
    ref.close()
    other.close()
