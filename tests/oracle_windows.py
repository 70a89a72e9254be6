"""Exact oracle references on windows of a large lattice (test helpers): the oracle runs
only small periodic windows, and a window's centre is exact as long as the steps taken on
it do not reach its wrapped edges."""
import numpy as np


def oracle_two_steps_at(win9, f_t, y, x):
    """Densities and momenta at node (y, x) after two oracle steps from the state f_t [c][i][y][x],
    exactly: a step depends on nodes up to 3 away, so each step-1 population of the 7 x 7
    neighbourhood comes from its own periodic 9 x 9 window (centre exact), and step 2 runs
    on a 9 x 9 window of those (its outer ring keeps the step-0 values, on which the centre
    does not depend).  Windows of one step only: a wider window run for two steps would
    step its wrapped, unphysical edges twice."""
    ny, nx = f_t.shape[2:]

    def window(f, yc, xc):
        ys = (np.arange(-4, 5) + yc) % ny
        xs = (np.arange(-4, 5) + xc) % nx
        return f[:, :, ys][:, :, :, xs]

    f1 = window(f_t, y, x).copy()
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            f1[:, :, 4 + dy, 4 + dx] = win9.run(window(f_t, y + dy, x + dx), 1)[:, :, 4, 4]
    f2 = win9.run(f1, 1)
    rho, mom = win9.moments(f2)
    return rho[:, 4, 4], mom[:, :, 4, 4]
