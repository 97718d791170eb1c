import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def rel_err(x, ref):
    """max|x - ref| / max(max|ref|, 1e-12), per tensor."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))), 1e-12))


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


def check_mlp_grads(orc, dims, params, x, g_out, gpu_gp, gpu_gx, tol, out_sigmoid=True,
                    tau=1e-6, errors=None):
    """Compare MLP parameter / input gradients with the FP64 oracle.

    A sample whose smallest ReLU input is within rounding of 0 (|z| < tau)
    can switch a unit in one precision and not in the other; its share of
    the parameter gradient is allowed as slack (twice its magnitude) and its
    input-gradient row is not compared.  errors (a dict, optional) receives
    each tensor's relative error.  Returns the number of such samples.
    """
    import numpy as np
    zmin = orc.mlp_min_abs_preact(dims, params, x)
    amb = np.nonzero(zmin < tau)[0]
    gp, gx = orc.mlp_bwd(dims, params, x, g_out, out_sigmoid)
    slack = np.zeros_like(gp)
    for s in amb:
        gps, _ = orc.mlp_bwd(dims, params, x[s:s + 1], g_out[s:s + 1], out_sigmoid)
        slack += 2 * np.abs(gps)
    offs = [0]
    for i in range(len(dims) - 1):
        offs += [offs[-1] + dims[i + 1] * dims[i], offs[-1] + dims[i + 1] * dims[i] + dims[i + 1]]
    for li, (a, b) in enumerate(zip(offs[:-1], offs[1:])):
        err = np.abs(np.asarray(gpu_gp[a:b], np.float64) - gp[a:b])
        lim = tol * max(np.max(np.abs(gp[a:b])), 1e-30) + slack[a:b]
        if errors is not None:
            errors[("W", "b")[li % 2] + str(li // 2 + 1)] = rel_err(gpu_gp[a:b], gp[a:b])
        assert np.all(err <= lim), (a, b, float(np.max(err - lim)), float(np.max(np.abs(gp[a:b]))))
    if gpu_gx is not None:
        keep = np.ones(x.shape[0], bool)
        keep[amb] = False
        e = rel_err(np.asarray(gpu_gx)[keep], gx[keep][:, :np.asarray(gpu_gx).shape[1]])
        if errors is not None:
            errors["g_x"] = e
        assert e < tol
    return len(amb)
