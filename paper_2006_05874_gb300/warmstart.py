"""Learned warm start of the adaptive IHS (an addition: the paper starts the
doubling of m at 1).

A small network (11 -> 64 -> 64 -> 1, tanh) maps cheap features of (A, nu) to
a prediction of log2 of the sketch size a cold run settles at; the solve then
starts at 2^(floor(prediction) - 1).  Features, network, training gradients
and the Adam step all run in the library's kernels (``ihs_probe_features``,
``ihs_mlp_*``, ``ihs_warm_start``); this module only loads the trained
parameters onto the device.  ``train_warmstart`` produces the parameter file.
"""
import json
import os

import numpy as np

WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_weights.json")


def load_params(path=WEIGHTS_PATH):
    """The trained flat parameter vector (float32 numpy) and the file's metadata."""
    with open(path) as f:
        doc = json.load(f)
    p = np.asarray(doc["params"], dtype=np.float32)
    meta = {k: v for k, v in doc.items() if k != "params"}
    return p, meta


class WarmStart:
    """Device copy of the trained parameters bound to a Context."""

    def __init__(self, ctx, path=WEIGHTS_PATH, params=None):
        import torch

        from . import ihs

        if params is None:
            params, self.meta = load_params(path)
        else:
            self.meta = {}
        nparam = ihs.load().ihs_mlp_num_params()
        if params.size != nparam:
            raise ValueError("parameter file holds %d values, the network has %d" % (params.size, nparam))
        self.ctx = ctx
        self.params = torch.as_tensor(np.ascontiguousarray(params, dtype=np.float32), device="cuda")

    def m0(self, A, nu, seed=None):
        """(initial sketch size, raw prediction of log2 m_settled)."""
        return self.ctx.warm_start(self.params, A, nu, seed)

    def solve(self, A, b, nu, x, tol=0.0):
        """Warm-started solve: sets m_init from the prediction, solves, restores m_init."""
        m0, pred = self.m0(A, nu)
        old = self.ctx.params.m_init
        self.ctx.set_params(m_init=m0)
        try:
            rep = self.ctx.solve(A, b, nu, x, tol=tol)
        finally:
            self.ctx.set_params(m_init=old)
        return rep, m0, pred
