"""Write tests/golden/config3_crop_oracle.npz: the FP64 CPU oracle's outputs on
the cropped config-3 problem (``workloads.config3_crop``: 8x8 PMUTs, a 32x32x16
N=4 primary box under a 16x16x96 N=6 secondary box, 6,510,658 nodes, 8000
steps of Algorithm 1).  Calls only ``oracle/`` and ``workloads/``; nothing here
comes from the CUDA path.  Takes about an hour on one core.

Stored (sample conventions of the oracle's run: callback n holds p^{n+1},
q^{n+1}):
  dt                the oracle's time step
  traces            [1][64][2000] receiver samples n = 3, 7, 11, ... (every
                    4th step: p^{4}, p^{8}, ...)
  q_steps, q        the modal coordinates q^{s} for s = 40, 80, ..., 8000,
                    shape [200][n_pmut * n_modes]
  e_steps, energy   the leapfrog energy 1/2 v.M v + 1/2 p^s.K p^{s+1} and the
                    semi-discrete coupled energy after s = 400, 800, ... steps
  p_nodes, p_final  p^{8000} at every 1009th node (node order of the oracle:
                    primary lattice then secondary, x fastest)

Usage: python tests/golden/make_config3_crop_oracle.py [nsteps]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import dgsem_oracle as O  # noqa: E402

TRACE_EVERY = 4
Q_EVERY = 40
E_EVERY = 400
NODE_STRIDE = 1009


def main(nsteps=8000, out=os.path.join(HERE, "config3_crop_oracle.npz")):
    t0 = time.time()
    w = W.config3_crop(nsteps=nsteps)
    P = O.OracleProblem(w)
    dt = P.stable_dt()
    drive = w.drive(dt, nsteps, 1)
    print(f"assembled {P.nh} nodes, nnz(K) = {P.K.nnz} in {time.time() - t0:.0f} s", flush=True)
    q_steps, q_rec, e_steps, e_rec = [], [], [], []

    def cb(n, p, pd, pdd, q, qd, qdd):
        s = n + 1
        if s % Q_EVERY == 0:
            q_steps.append(s)
            q_rec.append(q[:, 0].copy())
        if s % E_EVERY == 0:
            e_steps.append(s)
            e_rec.append(P.energy(p, pd, pdd, dt, q, qd, qdd)[:, 0])
            print(f"step {s}: E = {e_rec[-1]}  ({time.time() - t0:.0f} s)", flush=True)

    traces = P.run(nsteps=nsteps, dt=dt, drive=drive, batch=1, callback=cb)
    nodes = np.arange(0, P.nh, NODE_STRIDE)
    np.savez_compressed(out, dt=dt, nsteps=nsteps, trace_every=TRACE_EVERY,
                        traces=traces[:, :, TRACE_EVERY - 1::TRACE_EVERY],
                        q_steps=np.array(q_steps), q=np.array(q_rec),
                        e_steps=np.array(e_steps), energy=np.array(e_rec),
                        p_nodes=nodes, p_final=P.final_state["p"][nodes, 0])
    print(f"wrote {out} after {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 8000)
