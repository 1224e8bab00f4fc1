"""Helpers shared by the GPU parity tests."""
import numpy as np
import pytest


def gpu_package():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device (there is no CPU fallback)")
    import __graft_entry__ as g
    g.build()
    import paper_2603_07321_gb300 as P
    return P


def on_grid(x, bits=24):
    """Round coordinates to multiples of 2^-bits A, so that both the FP64 and
    the mixed (hi + lo) representation hold them exactly."""
    s = float(2 ** bits)
    return np.round(np.asarray(x) * s) / s


def force_error(f, f_ref):
    """max_i |F_i - F_ref_i| / rms_i |F_ref_i|"""
    scale = np.sqrt(np.mean(np.sum(f_ref ** 2, axis=1)))
    return np.max(np.linalg.norm(f - f_ref, axis=1)) / scale


def force_error_atom(f, f_ref):
    """max_i |F_i - F_ref_i| / max(|F_ref_i|, rms_i |F_ref_i|): the error of
    each atom's force relative to that force, with the rms force as the floor
    where a force is near zero"""
    fn = np.linalg.norm(f_ref, axis=1)
    scale = np.sqrt(np.mean(fn ** 2))
    return np.max(np.linalg.norm(f - f_ref, axis=1) / np.maximum(fn, scale))


def force_error_rms(f, f_ref):
    """rms_i |F_i - F_ref_i| / rms_i |F_ref_i|"""
    return np.sqrt(np.mean(np.sum((f - f_ref) ** 2, axis=1)) / np.mean(np.sum(f_ref ** 2, axis=1)))


def sorted_rows(counts, lst):
    return [sorted(lst[i, : counts[i]].tolist()) for i in range(len(counts))]
