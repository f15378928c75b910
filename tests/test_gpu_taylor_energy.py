"""Energy balance of the Taylor impact on the GPU paths (Sec. 2.1, Eq.
conservation3; the rigid wall is a reading, the paper has no contact).

Each path's own fields close the velocity-Verlet balance: the shadow energy
(kinetic energy less dt^2/8 sum |f|^2/m, plus the internal energy sum m e)
stays at its initial value once the work the wall removes is added back,
and the kinetic and internal energies follow the FP64 oracle's."""
import numpy as np
import pytest

import oracle
from paper_1901_07374_gb300 import tlsph
from parity import shadow_energy, taylor_energy_terms, taylor_energy_workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-3)])
def test_taylor_impact_energy_balance_gpu(precision, tol):
    w = taylor_energy_workload()
    g = tlsph.Simulation.from_workload(w, precision=precision)
    o = oracle.Simulation.from_workload(w)
    mass = w.specimen.vol * w.materials[0]["rho0"]
    E0 = shadow_energy(mass, w.dt, g.get("V"), g.get("FORCE"), g.get("ENERGY"))
    wall, worst, contact = 0.0, 0.0, None
    for k in range(w.steps):
        v_n, f_n = g.get("V"), g.get("FORCE")
        g.step(1)
        o.step(1)
        v, f, e = g.get("V"), g.get("FORCE"), g.get("ENERGY")
        dW = taylor_energy_terms(mass, w.dt, v_n, f_n, v, f)
        wall += dW
        if contact is None and dW > 1e-9 * E0:
            contact = k
        E = shadow_energy(mass, w.dt, v, f, e)
        if contact is None:
            assert E == pytest.approx(E0, rel=1e-12)
        worst = max(worst, abs(E + wall - E0) / E0)
        if k % 20 == 19:
            ke, ie = 0.5 * np.sum(mass[:, None] * v * v), np.sum(mass * e)
            ke_o, ie_o = 0.5 * np.sum(mass[:, None] * o["v"] ** 2), np.sum(mass * o["e"])
            assert abs(ke - ke_o) <= tol * E0 and abs(ie - ie_o) <= tol * E0, (k, ke, ke_o, ie, ie_o)
            d = g.diagnostics()        # the library's own reductions of the same sums
            assert d["kinetic_energy"] == pytest.approx(ke, rel=1e-9)
            assert d["internal_energy"] == pytest.approx(ie, rel=1e-9, abs=1e-12 * E0)
    assert contact is not None and wall > 0.02 * E0
    assert worst < 3e-3, worst
