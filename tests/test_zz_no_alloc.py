"""The allocation-free EAM entry point (ne_eam_energy_forces_noalloc).

It serves callers that cannot allocate device memory while they run -- an
engine that has reserved the device memory for its own pool, or a real-time
pipeline that forbids cudaMalloc after start-up.  Its scratch is a fixed
device array inside the library, shared by every call, so the test makes two
calls in a row (different sizes and lattices, so stale contents from the
first call would show) and compares each with ne_eam_energy_forces, the
entry point that allocates its buffers in a context, within the tolerances
of the GPU parity tests.  It passes alone in a fresh process and after the
other GPU tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_2201_04622_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2201_04622_gb300 import ne  # noqa: E402

DEV = torch.device("cuda:0")


def _eval(fn, *args):
    f = torch.zeros((args[2].shape[0], 3), dtype=torch.float64, device=DEV)
    e = torch.zeros(1, dtype=torch.float64, device=DEV)
    fn(*args, f=f, e=e)
    torch.cuda.synchronize()
    return float(e.item()), f.cpu().numpy()


def test_noalloc_matches_context_entry_point_on_two_calls_in_a_row():
    eam = ne.eam_params(**W.EAM_FE_LIKE)
    ctx = ne.ne_ctx_create(eam, 4096, 1)
    try:
        cases = [(O.BCC, W.A_BCC, 8, 0.12, 3), (O.FCC, W.A_FCC, 5, 0.1, 4)]
        for prec, e_tol, f_tol in [(ne.NE_FP64, 1e-10, 1e-10), (ne.NE_MIXED, 1e-6, 5e-5)]:
            for lat, a, n, amp, seed in cases:
                x0, box = O.create_crystal(lat, a, n, n, n)
                x = torch.tensor(W.displaced(x0, amp, seed), dtype=torch.float64, device=DEV)
                e1, f1 = _eval(ne.ne_eam_energy_forces_noalloc, eam, prec, x, box)
                e2, f2 = _eval(ne.ne_eam_energy_forces, ctx, prec, x, box)
                assert e1 == pytest.approx(e2, rel=e_tol)
                assert np.linalg.norm(f1 - f2) / np.linalg.norm(f2) < f_tol
    finally:
        ne.ne_ctx_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_limit():
    eam = ne.eam_params(**W.EAM_FE_LIKE)
    x0, box = O.create_crystal(O.BCC, W.A_BCC, 11, 11, 11)  # 2662 atoms > 2048
    x = torch.tensor(x0, dtype=torch.float64, device=DEV)
    e = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(ne.NeError, match="NE_ENOMEM"):
        ne.ne_eam_energy_forces_noalloc(eam, ne.NE_FP64, x, box, e=e)
