"""Pins for the oracle's density of states (Sec. 3): in the complete limit the columns' Lorentzian-broadened
weights add up to the broadened spectrum of the dense generalized eigenproblem, sum_n eta / pi / ((E - E_n)^2
+ eta^2) (each state's weights over all columns sum to one: Phi^T S Phi = I); for a truncated column the DOS
term equals -(1/pi) Im sum_i G_ij(z) S_ji from the Green's function column itself."""
import numpy as np
import pytest
import scipy.linalg

from oracle import mka, sk as osk, system as osys
from synth import WORKLOADS, random_symmetric_pair, workload_positions


@pytest.mark.parametrize("m,seed", [(12, 0), (20, 1)])
def test_complete_limit_is_the_broadened_spectrum(m, seed):
    H, S = random_symmetric_pair(m, seed)
    E_n = scipy.linalg.eigh(H, S, eigvals_only=True)
    eps, w = [], []
    for j in range(m):
        c = mka.solve_column(H, S, j, m, m)
        eps.append(c.eps)
        w.append(c.w)
    grid = np.linspace(E_n.min() - 1, E_n.max() + 1, 37)
    eta = 0.07
    ref = np.array([np.sum(eta / np.pi / ((E - E_n) ** 2 + eta ** 2)) for E in grid])
    np.testing.assert_allclose(mka.dos(np.concatenate(eps), np.concatenate(w), grid, eta), ref, rtol=1e-11, atol=1e-11)


def test_column_term_is_minus_im_trace_of_G_S():
    w_ = WORKLOADS["diamond512"]
    pos, box = workload_positions(w_)
    res = osys.solve_atoms(pos, box, w_.sk, w_.R, [17], w_.p, w_.q, keep_full=True)
    r = res[0]
    _, Sc = osk.cluster_matrices(pos, box, r.cluster, w_.sk)
    m = Sc.shape[0]
    eta = 0.05
    for c in r.cols:
        for E in (-3.0, 0.7, 2.5):
            g = mka.greens_column(c, complex(E, eta), np.arange(m))      # G_ij for all i of the cluster
            ref = -np.imag(g @ Sc[c.j, :]) / np.pi
            assert abs(mka.dos(c.eps, c.w, [E], eta)[0] - ref) < 1e-12
