"""FP64 CPU oracle of the density-fitted particle-particle ladder.

TEST INFRASTRUCTURE ONLY: imported by tests/ and the benchmark's CPU
baseline; the GPU library never imports it and it imports nothing from it.

The ladder is the linear term of the doubles residual of H + [H, T] (Sec. 2.2)
in which the two-electron integral has all four indices virtual:

    R^{ab}_{kl} = sum_{e,f} <ab|ef> T^{ef}_{kl} = sum_{e,f} (ae|bf) T^{ef}_{kl}

with the density-fitted chemist integral (ae|bf) = sum_Q B_Qae B_Qbf
(Sec. 2.1 for <pq|rs> = (pr|qs)).  Indices: k, l holes (core or active),
a, b, e, f virtual.  Written from the definition: the integrals, then the
contraction, each one library call.
"""
from __future__ import annotations

import numpy as np


def ladder_vvvv(Bvv, T):
    """R[k,l,a,b] = sum_{e,f} (ae|bf) T[k,l,e,f] for Bvv [Q,v,v], T [h,h,v,v].

    One virtual a at a time: the integrals (ae|bf) for that a ([b, e, f]),
    then their contraction with T, so memory stays at v^3 numbers."""
    nh, v, X = T.shape[0], T.shape[2], Bvv.shape[0]
    R = np.zeros((nh, nh, v, v))
    Tm = T.reshape(nh * nh, v * v)  # [(k,l), (e,f)]
    Bm = Bvv.reshape(X, v * v)      # [Q, (b,f)]
    for a in range(v):
        V_a = (Bvv[:, a, :].T @ Bm).reshape(v, v, v)  # [e, b, f] = (ae|bf)
        Vt = V_a.transpose(0, 2, 1).reshape(v * v, v)  # [(e,f), b]
        R[:, :, a, :] = (Tm @ Vt).reshape(nh, nh, v)
    return R


def ladder_element(Bvv_a, Bvv_b, T_kl):
    """One element R[k,l,a,b] from the factor columns B[:, a, :], B[:, b, :]
    ([Q, v] each) and the amplitude block T[k, l] ([v, v])."""
    V_ab = Bvv_a.T @ Bvv_b  # [e, f] = (ae|bf)
    return float(np.sum(V_ab * T_kl))
