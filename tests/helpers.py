"""Shared test helpers: record conversion and the parity comparisons used by
the GPU tests (the oracle is the reference; margins explain mismatches)."""
import numpy as np

import oracle

C_LIGHT = 299792458.0


def rec_to_paths(rec: np.ndarray) -> np.ndarray:
    """uint32 [n, 8] path records -> oracle PATH_DTYPE."""
    rec = np.asarray(rec, np.uint32).reshape(-1, 8)
    p = np.zeros(len(rec), oracle.PATH_DTYPE)
    p["tx"] = rec[:, 0]
    p["rx"] = rec[:, 1]
    p["depth"] = rec[:, 2] & 15
    p["face"] = rec[:, 3:7]
    p["ray"] = rec[:, 7]
    p["flag"] = rec[:, 2] >> 8
    return p


def keys(p) -> list:
    return [tuple(r) for r in oracle.key_fields(p)]


def compare_candidates(gpu_unique, orc_cands, ray_marg, rx_rows=None):
    """Discovery parity.  Every oracle candidate found by a ray whose outcome
    is outside the margin must be on the GPU; every GPU candidate must be an
    oracle candidate or come from a ray the oracle flags as marginal at or
    before the candidate's depth.  ray_marg rows are transmitters, or, for
    backward discovery, receivers: rx_rows maps a receiver id to its row.
    Returns a summary dict."""
    ou = oracle.dedup(orc_cands)
    okeys = keys(ou)
    oflag = dict(zip(okeys, ou["flag"].tolist()))
    gkeys = keys(gpu_unique)
    gset = set(gkeys)
    missing = [k for k, f in oflag.items() if f == 0 and k not in gset]
    extra_bad = []
    extra_marg = 0
    for k, p in zip(gkeys, gpu_unique):
        if k in oflag:
            continue
        row = int(p["tx"]) if rx_rows is None else rx_rows[int(p["rx"])]
        j, depth = int(p["ray"]), int(p["depth"])
        if ray_marg[row, j] <= depth:
            extra_marg += 1
        else:
            extra_bad.append(k)
    return dict(n_gpu=len(gset), n_orc=len(okeys), missing=missing, extra_bad=extra_bad,
                extra_marginal=extra_marg,
                oracle_marginal=sum(1 for f in oflag.values() if f != 0))


def compare_acceptance(os_, gpu_paths, eps_abs=1e-4, eps_rel=0.0):
    """Acceptance parity on the GPU's own candidate list."""
    acc_o, marg_o = oracle.validate(os_, gpu_paths, eps_abs=eps_abs, eps_rel=eps_rel)
    acc_g = (gpu_paths["flag"] & 1).astype(bool)
    diff = acc_o != acc_g
    bad = np.nonzero(diff & (marg_o == 0))[0]
    return dict(n=len(gpu_paths), n_acc_gpu=int(acc_g.sum()), n_acc_orc=int(acc_o.sum()),
                n_diff=int(diff.sum()), n_diff_unflagged=len(bad), bad=bad)


def compare_field(a_g, tau_g, fd_g, a_o, tau_o, fd_o, amp_rel=1e-4, phase_rad=1e-3):
    """Element-wise field parity: amplitude 1e-4 relative, phase 1e-3 rad."""
    amp_err = np.abs(np.abs(a_g) - np.abs(a_o)) / np.maximum(np.abs(a_o), 1e-300)
    ph_err = np.abs(np.angle(a_g * np.conj(a_o)))
    tau_err = np.abs(tau_g - tau_o) / np.maximum(tau_o, 1e-300)
    fd_err = np.abs(fd_g - fd_o) / np.maximum(1.0, np.abs(fd_o))
    return dict(amp=float(amp_err.max(initial=0)), phase=float(ph_err.max(initial=0)),
                tau=float(tau_err.max(initial=0)), fd=float(fd_err.max(initial=0)),
                ok=bool((amp_err <= amp_rel).all() and (ph_err <= phase_rad).all()
                        and (tau_err <= 1e-12).all() and (fd_err <= 1e-9).all()))


def compare_accepted(os_, gpu_acc, orc_cands, ray_marg):
    """Parity of a final accepted path set (discovery + acceptance) with the
    oracle's on the same rays: the oracle deduplicates its candidates and
    accepts them itself.  An oracle-accepted path may be missing on the GPU
    only if the oracle flags its discovery or acceptance as marginal; a GPU
    path the oracle does not accept must be flagged: by the GPU (reflection
    point within the margin), by the oracle's acceptance margin, or by the
    oracle's discovery margin of the ray that found it.  Returns a summary
    dict."""
    ou = oracle.dedup(orc_cands)
    acc_o, marg_o = oracle.validate(os_, ou)
    okeys = keys(ou)
    o_acc = {k: (int(f) != 0 or int(m) != 0)
             for k, a, f, m in zip(okeys, acc_o, ou["flag"], marg_o) if a}
    o_cand_marg = {k: int(m) != 0 for k, a, m in zip(okeys, acc_o, marg_o) if not a}
    gkeys = keys(gpu_acc)
    gset = set(gkeys)
    missing = [k for k, flagged in o_acc.items() if not flagged and k not in gset]
    extra_bad, extra_flagged = [], 0
    for k, p in zip(gkeys, gpu_acc):
        if k in o_acc:
            continue
        flagged = bool(int(p["flag"]) & 2) or o_cand_marg.get(k, False) or \
            ray_marg[int(p["tx"]), int(p["ray"])] <= int(p["depth"])
        if flagged:
            extra_flagged += 1
        else:
            extra_bad.append(k)
    return dict(n_gpu=len(gset), n_orc=len(o_acc), missing=missing, extra_bad=extra_bad,
                extra_flagged=extra_flagged,
                missing_flagged=sum(1 for k, f in o_acc.items() if f and k not in gset))
