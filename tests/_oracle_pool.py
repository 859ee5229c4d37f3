"""Oracle work for one source of the 3-D apply workload, run in a spawn-context process
pool by the GPU parity tests (test infrastructure: imports only the oracle, the input
generators and numpy).  For source a: the oracle's own state solve, its tangent, J p at
the receivers and J_a^T y_a over all nodes for the given columns."""
import numpy as np


def source_reference(args):
    """args: (source index, p columns [N, c], y_a columns [n_rec, c])."""
    a, p, y = args
    import oracle as O
    from paper_2609_14982_b300 import workloads as W
    wl = W.config3()
    g = wl.grid
    _, G, _ = O.metric(g)
    k = int(wl.src[a])
    T, cyc = O.eik_forward(g, wl.s, k)
    t = O.build_tangent(g, G, T, wl.s, k)
    jp = O.J([t], wl.s, wl.rec, p)[0]
    jt = O.JT([t], wl.s, wl.rec, y[None], sum_sources=False)[0]
    return a, T, t.label, t.perm, t.level_ptr, jp, jt
