"""The oracle's collision velocity u = (j + (n g + C)/2)/n: the velocity of
the second-order forcing in the collision (Eq. SMDB), formed from the
oracle's populations and its fields C (Eq. campoc) of the same state.  The
oracle's moments() return the field velocity v of reading R7 instead, which
equals u at a steady state (tests/test_oracle_linear.py pins that)."""
import numpy as np


def collision_velocity(oracle_mod, o, g):
    c, _ = oracle_mod.velocities()
    f = o.populations()
    n = f.sum(axis=0)
    j = np.einsum("qzyx,qa->azyx", f, c.astype(float))
    _, C, _ = o.fields()
    with np.errstate(invalid="ignore", divide="ignore"):       # solid planes: n = 0
        return np.array([(j[a] + 0.5 * (n * g[a] + C[a])) / n for a in range(3)])
