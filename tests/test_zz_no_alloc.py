"""lbs_moments_static, the entry point for callers that cannot allocate device
memory where they need moments (it keeps its scratch in a fixed array inside the
library): its profiles must equal those of lbs_profiles for the same state, on
two calls in a row with different states, so nothing stale survives in the shared
scratch between calls.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads as W
from tests._pair import profile_errors

pytestmark = pytest.mark.gpu

RAGGED = dict(Qx=6, Qy=5, Qz=7, N_eq=4, Nz=37, A=0.9, Kn=0.3, u_w=0.4, T_w=1.0, Pr=2.0 / 3.0,
              visc_law=1, visc_param=0.5239)


# the tolerances of the parity tests: 1e-12 (FP64 storage), 2e-5 (FP32 storage)
@pytest.mark.parametrize("params,precision,tol", [(RAGGED, 0, 1e-12), (W.C2, 1, 2e-5)])
def test_static_moments_match_profiles(params, precision, tol):
    import torch

    from paper_1702_01335_gb300 import PROFILE_NAMES, Instance, Solver
    torch.cuda.set_device(0)
    s = Solver(Instance(**params), precision=precision)
    st = s.torch_stream()
    Nz, Q = params["Nz"], Instance(**params).Q
    # the whole stored state (deviations, then the FP32 residuals); the call reads the
    # deviations at its start
    f_dev = torch.empty(s.state_bytes(), dtype=torch.uint8, device="cuda")
    out = torch.empty((14, Nz), dtype=torch.float64, device="cuda")
    free = []
    for call in range(2):
        s.step(7 + 5 * call)
        s.get_state_device(0, f_dev.data_ptr())
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        s.moments_static(0, f_dev.data_ptr(), out.data_ptr())
        with torch.cuda.stream(st):
            got = out.cpu().numpy()
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ref = s.profiles(0)
        errs = profile_errors(dict(zip(PROFILE_NAMES, got)), ref)
        assert max(errs.values()) < tol, (call, errs)
    # no device memory taken by the calls themselves (the first call may load the module's
    # scratch array, which is part of the library image; the second call must not grow it)
    assert free[2] == free[3], free
    s.close()


def test_static_moments_rejects_oversize():
    """ceil(8192 / 512) * 2048 cells exceeds the fixed scratch: rejected on the host."""
    import torch

    from paper_1702_01335_gb300 import Instance, LbsError, Solver
    p = dict(W.C3, Nz=2048)
    s = Solver(Instance(**p), precision=1)
    f_dev = torch.zeros((p["Nz"], Instance(**p).Q), dtype=torch.float32, device="cuda")
    out = torch.zeros((14, p["Nz"]), dtype=torch.float64, device="cuda")
    with pytest.raises(LbsError) as e:
        s.moments_static(0, f_dev.data_ptr(), out.data_ptr())
    assert e.value.status == 1
    s.close()
