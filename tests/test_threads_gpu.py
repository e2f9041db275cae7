"""Contexts driven from two host threads at once: every kernel-attribute and
SM-count cache of the library is per device and behind a lock, so both
threads' first launches (which set the attributes) may race; both volumes
must still match the oracle."""
import threading

import numpy as np
import pytest
import torch

from paper_1910_08498_gb300 import _lib as L
from paper_1910_08498_gb300 import inputs
from tests.helpers import A32, ALPHA, TOL_F32, oracle_insert, rel_err

pytestmark = pytest.mark.gpu


def _worker(S, seed, cfg, out, key):
    try:
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        img, rot = inputs.make_batch(S, 48, seed)
        with torch.cuda.stream(stream):
            ctx = L.fr_create(S, A32, ALPHA, 0, 10000)
            try:
                if cfg >= 0 and not L.fr_config_valid(ctx, cfg):
                    cfg = -1
                L.fr_set_options(ctx, tuning=0, forced_config=cfg)
                img_d, rot_d = img.cuda(), rot.cuda()
                for _ in range(2):
                    L.fr_insert(ctx, img_d, rot_d, stream=stream)
                D = S + 1
                V = torch.empty(D ** 3, dtype=torch.complex64, device="cuda")
                W = torch.empty(D ** 3, dtype=torch.float32, device="cuda")
                L.fr_finalize(ctx, V, W, stream=stream)
                stream.synchronize()
                out[key] = (img, rot, V.cpu().numpy().astype(np.complex128),
                            W.cpu().numpy().astype(np.float64), L.fr_last_device_error(ctx))
            finally:
                L.fr_destroy(ctx)
    except Exception as e:  # reported by the main thread
        out[key] = e


@pytest.mark.parametrize("cfgs", [(-1, -1), (13, 41), (-1, 4)])
def test_two_host_threads(cfgs):
    out = {}
    th = [threading.Thread(target=_worker, args=(S, 300 + S, c, out, i))
          for i, (S, c) in enumerate(zip((32, 48), cfgs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for i, S in enumerate((32, 48)):
        r = out[i]
        assert not isinstance(r, Exception), r
        img, rot, V, W, err = r
        assert err == L.FR_OK
        Vr, Wr, _ = oracle_insert(S, [(img, rot), (img, rot)])
        assert rel_err(V, Vr) <= TOL_F32 and rel_err(W, Wr) <= TOL_F32
