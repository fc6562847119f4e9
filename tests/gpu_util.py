"""Helpers for the GPU parity tests: device buffers through torch, calls
through the C ABI binding."""

import numpy as np
import torch

import synth


def lib():
    from paper_2604_04696_gb300 import _build
    _build.build()
    from paper_2604_04696_gb300 import gpir
    return gpir


def to_dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).cuda()


def to_host(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


class DbHandle:
    def __init__(self, g, db_np, N, primes, path_mask=0, on_device=True):
        self.g = g
        self.params = g.gpir_params_create(N, list(primes))
        self.D0, self.D1 = db_np.shape[0], db_np.shape[1]
        self.L, self.N = len(primes), N
        if on_device:
            t = to_dev(db_np)
            self.h = g.gpir_db_upload(self.params, self.D0, self.D1, t, True, path_mask)
            del t
        else:
            self.h = g.gpir_db_upload(self.params, self.D0, self.D1, np.ascontiguousarray(db_np), False, path_mask)

    def rowsel(self, ct_dev: torch.Tensor, B: int, path: int, out=None) -> torch.Tensor:
        if out is None:
            out = torch.full((B, self.D1, 2, self.L, self.N), -1, dtype=torch.int32, device="cuda")
        self.g.gpir_rowsel_batch(self.h, B, ct_dev, out, path)
        torch.cuda.synchronize()
        self.g.gpir_sync(None, 20000)
        return out

    def close(self):
        self.g.gpir_db_free(self.h)
        self.g.gpir_params_destroy(self.params)


def make_problem(seed, B, D0, D1, L, N, primes):
    ct = synth.ct_tensor(seed, B, D0, L, N, primes)
    db = synth.db_tensor(seed, D0, D1, L, N, primes)
    return ct, db
