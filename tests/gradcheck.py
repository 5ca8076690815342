"""The bound the GPU's global gradients (dL/dD_L, dL/dD_T, dL/dlifetime) are held to.

Each global gradient is a sum over depos of per-depo chain-rule terms (Fig. 2's drift with
sigma = sqrt(2 D t_d) and Q' = Q exp(-t_d / tau)):
    dL/dD_L = sum_i dL/dsigma_L,i  sigma_L,i / (2 D_L)
    dL/dD_T = sum_i dL/dsigma_T,i  sigma_T,i / (2 D_T)
    dL/dtau = sum_i dL/dQ_i  Q_i t_d,i / tau^2
Terms of both signs cancel, so a per-term relative error e gives the sum an error of at most
e * sum_i |T_i|: relative to the sum, e times its condition number sum_i |T_i| / |sum_i T_i|.
The per-term error allowed is the per-output tolerance of the gradients (1e-5), so the sum
is held to 1e-5 * sum_i |T_i|, with the terms T_i taken from the FP64 oracle.
"""
import numpy as np

TERM_REL = 1e-5


def global_terms(prm, depos, ref):
    """The oracle's per-depo terms of the three global sums (ref: oracle depo_grads)."""
    td = np.asarray(depos.td, np.float64)
    q = np.asarray(depos.q, np.float64)
    out = {}
    sL = np.sqrt(2.0 * prm.DL_cm2_s * 1e-4 * td)
    sT = np.sqrt(2.0 * prm.DT_cm2_s * 1e-4 * td)
    out["DL"] = np.asarray(ref["sigma_L"]) * sL / (2.0 * prm.DL_cm2_s) if prm.DL_cm2_s > 0 else 0 * td
    out["DT"] = np.asarray(ref["sigma_T"]) * sT / (2.0 * prm.DT_cm2_s) if prm.DT_cm2_s > 0 else 0 * td
    out["lifetime"] = np.asarray(ref["q"]) * q * td / prm.lifetime_us ** 2
    return out


def assert_globals_close(got, ref, prm, depos, what=""):
    """|GPU - oracle| <= TERM_REL * sum_i |T_i| for each global gradient; returns the errors
    relative to the sums, and the sums' condition numbers."""
    terms = global_terms(prm, depos, ref)
    report = {}
    for k in ("DL", "DT", "lifetime"):
        t = terms[k]
        a, b = float(got[k].cpu()), float(ref[k])
        mag = float(np.abs(t).sum())
        # the oracle's global is the sum of its own terms (FP64 rounding only)
        assert abs(float(t.sum()) - b) <= 1e-9 * mag + 1e-300, (what, k, float(t.sum()), b)
        bound = TERM_REL * mag
        assert abs(a - b) <= bound, "%s %s: |%.9e - %.9e| = %.3e > %.3e (cond %.1f)" % (
            what, k, a, b, abs(a - b), bound, mag / max(abs(b), 1e-300))
        report[k] = (abs(a - b) / max(abs(b), 1e-300), mag / max(abs(b), 1e-300))
    return report
