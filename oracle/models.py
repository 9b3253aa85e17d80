"""Builds oracle models from the workload descriptions (input marshalling only; test infrastructure)."""
import oracle
from workloads import WORKLOADS, cubic_cell


def oracle_model(name, n, pbc=None, dipolar=False, build=True, **override):
    w = dict(WORKLOADS[name])
    w.update(override)
    m = oracle.Model(n, pbc if pbc is not None else w["pbc"], cubic_cell(), w["pos"], w["mu"])
    for k, J in enumerate(w["shells"]):
        if J != 0.0:
            m.add_shell_exchange(k + 1, J)
    if w["dmi"]:
        shell, kind, D = w["dmi"]
        m.add_dmi(shell, kind, D)
    m.set_zeeman(w["B"])
    if w["K"]:
        K, axis = w["K"]
        for s in range(len(w["pos"])):
            m.set_anisotropy(s, K, axis)
    m.set_dipolar(dipolar)
    if build:
        m.build()
    return m, w
