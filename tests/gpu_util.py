"""Helpers shared by the GPU parity tests: run the CUDA library through its
C ABI (via the binding) and compare with the CPU oracle."""
import numpy as np
import pytest
import torch

import cases

FIELDS = ("u", "v", "w", "alpha", "T", "p")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2209_09671_gb300 as P
    try:
        P.load()
    except RuntimeError as e:   # the library must be built on a GPU machine
        pytest.fail(str(e))
    return P


def gpu_step(P, prm, state, step_index=0, dt=0.0, nsteps=1, stream=True):
    """Steps through the C ABI.  On a stream of its own (the default) every
    pressure solve runs as a CUDA graph with its stopping test on the
    device; stream=False uses the legacy default stream, which cannot be
    captured, so the solves run as eager launches with the host loop."""
    st = torch.cuda.Stream() if stream else torch.cuda.current_stream()
    with torch.cuda.stream(st):
        solver = P.Solver(prm, stream=st)
        dev = P.to_device(state, prm.precision == cases.MIXED)
        infos = []
        for n in range(nsteps):
            infos.append(solver.fvm_step(dev, step_index + n, dt))
    torch.cuda.synchronize()
    host = {k: dev[k].double().cpu().numpy() for k in FIELDS}
    solver.close()
    return host, infos


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.linalg.norm(a)
    return np.linalg.norm(a - b) / nb
