"""The worker-process oracle runs used by the whole-trajectory GPU tests equal direct runs."""
import numpy as np

import oracle
from oracle_pool import labels_digest, run_all
from paper_1403_0240_gb300 import synth


def test_pool_trajectories_equal_direct_runs():
    specs = [("batch", 3, 1000), ("served", ("pc2d", 128, 7 * 128 + 4), 4)]
    out = run_all(specs, 4)
    for spec, (traj, n_ref, S_ref, Q_ref) in zip(specs, out):
        w = synth.batch_disk(3, seed0=1000) if spec[0] == "batch" else synth.served_job(spec[1], 4)
        p = oracle.make_params(w.image, w.labels0, w.model, w.connectivity, w.lam, w.cutoff, w.ps_radius)
        run = oracle.Run(p, w.image, w.labels0)
        for t in range(4):
            s, _ = run.step()
            assert traj[t][:5] == (s["n_particles"], s["n_candidates"], s["n_accepted"], s["mode_used"],
                                   s["converged"])
            assert traj[t][5] == labels_digest(run.L)
        n, S, Q = oracle.stats(p, w.image, run.L)
        assert np.array_equal(n, n_ref) and np.array_equal(S, S_ref) and np.array_equal(Q, Q_ref)
