import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300); parity tests of the CUDA path")
    config.addinivalue_line("markers", "slow: CPU test that takes more than ~10 s")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.lib()
    return oracle


@pytest.fixture(scope="session")
def om():
    """The CUDA library's binding; GPU tests fail loudly without a device."""
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    from paper_1410_1921_gb300 import build
    build.build()
    import paper_1410_1921_gb300 as P
    P.lib()
    return P


def recon_args(cfg):
    """(seed, shape, ...) of a synthetic.Recon for the oracle's reconstruct."""
    return (cfg.seed, cfg.shape, cfg.dx_nm, cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm, cfg.dmax_nm,
            cfg.porosity, cfg.xi, cfg.p0, cfg.dist, cfg.max_trials)


def recon_params(P, cfg):
    return P.recon_params(cfg.mean_nm, cfg.sd_nm, cfg.dmin_nm, cfg.dmax_nm, cfg.porosity, cfg.xi,
                          cfg.p0, cfg.dist, cfg.max_trials)
