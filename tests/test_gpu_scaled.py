"""GPU batched KM with a single scaling factor (the approximate variant):
the assignment is optimal for floor(C/s) (bit-exact against the oracle on
the scaled costs) and its true cost lies within the a-priori bound."""
import numpy as np
import pytest
import torch

from paper_2005_01182_gb300 import otassign as ot
from paper_2005_01182_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scale", [1, 3, 64, 4096])
def test_scaled_optimal_on_scaled_costs(oracle_mod, ctx, scale):
    cases = [W.grid_sqdist(300, grid=64, seed=3), W.uniform_costs(500, 520, seed=4),
             W.shapes_sqdist(700, seed=5), W.pixel_sqdist(1200, seed=6), W.grid_sqdist(5000, grid=560, seed=8)]
    for C in cases:
        n = C.shape[0]
        for dev in (True, False):
            Ct = torch.from_numpy(C).cuda() if dev else torch.from_numpy(C)
            r, c, bound = ot.ot_assign_solve_scaled(ctx, Ct, scale)
            torch.cuda.synchronize()
            a = r.cpu().numpy()
            assert len(set(a.tolist())) == n
            Cs = np.floor_divide(C, scale).astype(np.int32)
            opt_scaled = oracle_mod.km(Cs)[1] if n <= 1200 else None
            if opt_scaled is not None:
                assert int(Cs[np.arange(n), a].astype(np.int64).sum()) == opt_scaled
            true = int(c.cpu().item())
            assert true == int(C[np.arange(n), a].astype(np.int64).sum())
            assert bound == n * (scale - 1)
            if n <= 1200:
                opt = oracle_mod.km(C)[1]
                assert opt <= true <= opt + bound
                if scale == 1:
                    assert true == opt
