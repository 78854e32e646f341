"""Shared helpers of the GPU parity tests (comparison rules, uploads)."""
import numpy as np

RENDER_TOL = 2e-4     # max abs error per RGBA channel against the FP64 oracle
STOP_EPS = 5e-5       # early-exit band: an FP32 march may stop anywhere in it


def render_error(got: np.ndarray, ref: dict):
    """Per-pixel max channel error against the oracle.

    A ray whose FP64 opacity passes alpha_stop within STOP_EPS has several
    correct results (an FP32 march can stop a sample earlier or later); for
    such rays the error is the smallest against the oracle's states at
    alpha_stop - eps, alpha_stop and alpha_stop + eps.
    """
    g = got.astype(np.float64)
    e_mid = np.abs(g - ref["rgba"]).max(axis=-1)
    e_lo = np.abs(g - ref["lo"]).max(axis=-1)
    e_hi = np.abs(g - ref["hi"]).max(axis=-1)
    amb = ref["nsamp"][..., 0] != ref["nsamp"][..., 2]
    err = np.where(amb, np.minimum(e_mid, np.minimum(e_lo, e_hi)), e_mid)
    return err, amb


def sample_bounds(ref: dict):
    ns = ref["nsamp"].astype(np.int64)
    return int(ns[..., 0].sum()), int(ns[..., 2].sum())
