"""The paper's §6 convection-diffusion family in the oracle (context for Table 1, which is not pinned:
the viscosity mu and the random right-hand side are not given).

With mu = 1 and p = 2 the Fourier slice k = 0 of A (A^(1) + A^(2)) is a convection-diffusion matrix of
order n whose condition number grows like n^2 (~4e5 at n = 1000; the slice k = 1, A^(1) - A^(2), is the
pure convection band, ~1e3); unpreconditioned restarted tGMRES(10), tFOM(10) and
TBAS(10) then stall far above the paper's 1e-6, whereas Table 1 reports convergence in 11-66 iterations.
"""
import numpy as np

from oracle import krylov as kr, tubal as tb, tproduct as tp
from paper_2405_09233_gb300 import inputs


def test_convection_diffusion_slices_are_ill_conditioned():
    pr = inputs.convdiff_problem(1000, 3, 2, mu=1.0, seed=0)
    Ah = tp.dft3(pr.A)
    kappa = [np.linalg.cond(Ah[:, :, k]) for k in range(2)]
    assert kappa[0] > 1e5 and kappa[1] > 1e2


def test_restarted_methods_stall_on_the_paper_example():
    pr = inputs.convdiff_problem(1000, 3, 2, mu=1.0, seed=0)
    g = kr.restarted_solve("gmres", pr.A, pr.B, pr.C, m=10, tol=1e-6, max_restarts=3)
    f = kr.restarted_solve("fom", pr.A, pr.B, pr.C, m=10, tol=1e-6, max_restarts=3)
    t = tb.tbas(pr.A, pr.B, pr.C, m=10, tol=1e-6, max_restarts=3)
    assert g.status == f.status == t.status == "not_converged"
    assert g.true_res[-1] > 0.5 * g.normC           # GMRES residuals never increase but barely move
    assert all(b <= a * (1 + 1e-12) for a, b in zip(g.history, g.history[1:]))
