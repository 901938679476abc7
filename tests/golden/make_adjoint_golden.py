"""Writes adjoint_porous_crop32x32x16.json: the FP64 tangent of the soft-
occupancy oracle (oracle/soft.py, dual numbers) for the 32x32x16 porous
crop after 2000 steps, the reference for the GPU adjoint test.  Calls only
the oracle and the seeded input generators.

    python tests/golden/make_adjoint_golden.py
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.soft import SoftLBE, from_ids  # noqa: E402
from paper_1907_04732_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "adjoint_porous_crop32x32x16.json")


def case():
    w = wl.porous_crop()
    chi, label = from_ids(w.ids)
    return w, chi, label


def chi_nodes(w):
    """A fluid node next to the porous electrode and an interface node of it."""
    flat = w.ids.reshape(-1)
    near = np.zeros(flat.size, dtype=bool)
    for s in (-1, 1):
        for ax in range(3):
            near |= (np.roll(w.ids, s, axis=ax) != 0).reshape(-1)
    fluid = int(np.flatnonzero((flat == 0) & near)[40])
    iface = int(np.flatnonzero((flat == 1) & (np.roll(w.ids, -1, axis=0).reshape(-1) == 0))[30])
    return fluid, iface


def directions(w, chi):
    rng = np.random.Generator(np.random.PCG64(wl.SEED + 5))
    fluid, iface = chi_nodes(w)
    e_f, e_i = np.zeros(chi.size), np.zeros(chi.size)
    e_f[fluid] = 1.0
    e_i[iface] = 1.0
    return {"psi2": {"dpsi": [0.0, 1.0]}, "debye": {"ddebye": 1.0}, "D+": {"dD": [1.0, 0.0]},
            "D-": {"dD": [0.0, 1.0]}, "chi_random": {"dchi": rng.standard_normal(chi.size)},
            "chi_fluid_node": {"dchi": e_f}, "chi_interface_node": {"dchi": e_i}}


def one(name):
    w, chi, label = case()
    m = SoftLBE(w.shape, w.periodic, label.reshape(w.ids.shape), w.bjerrum, e_app=w.e_app)
    q, dq = m.tangent(w.psi, w.debye, w.D, chi, w.steps, **directions(w, chi)[name])
    return name, q.tolist(), dq.tolist()


def main():
    w, chi, _ = case()
    names = list(directions(w, chi))
    with mp.get_context("spawn").Pool(min(len(names), os.cpu_count() or 1)) as pool:
        res = pool.map(one, names)
    fluid, iface = chi_nodes(w)
    out = {"source": "oracle/soft.py dual-number tangent, FP64",
           "workload": w.name, "shape": list(w.shape), "periodic": list(w.periodic), "psi": list(w.psi),
           "debye": w.debye, "bjerrum": w.bjerrum, "D": list(w.D), "steps": w.steps,
           "chi_random_seed": wl.SEED + 5, "chi_fluid_node": fluid, "chi_interface_node": iface,
           "Q": res[0][1], "dQ": {name: dq for name, _, dq in res}}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
