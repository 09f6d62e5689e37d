"""Argument checks of the Python binding that run before any library call (no GPU needed)."""
import numpy as np
import pytest
import torch

from paper_1709_06955_gb300 import probesim


def _args(nq=3, n=10, kmax=4):
    return (torch.zeros((nq, n), dtype=torch.float32), list(range(nq)), [2] * nq, kmax,
            torch.zeros((nq, kmax), dtype=torch.int32), torch.zeros((nq, kmax), dtype=torch.float32))


@pytest.mark.parametrize("bad", ["nodes", "ks", "ids_shape", "vals_dtype", "scores_dtype", "host_memory"])
def test_noalloc_binding_rejects_mismatched_buffers(bad):
    scores, nodes, ks, kmax, ids, vals = _args()
    if bad == "nodes":
        nodes = nodes[:2]
    elif bad == "ks":
        ks = ks + [1]
    elif bad == "ids_shape":
        ids = torch.zeros((3, kmax + 1), dtype=torch.int32)
    elif bad == "vals_dtype":
        vals = torch.zeros((3, kmax), dtype=torch.float64)
    elif bad == "scores_dtype":
        scores = scores.half()
    # host_memory: every shape and type is right, but the buffers are not CUDA memory
    with pytest.raises(ValueError):
        probesim.topk_select_noalloc(scores, nodes, ks, kmax, ids, vals)
    assert np.all(ids.numpy() == 0)
