"""Several ranks (gloo, world size 2, on the CPU): each rank processes its
own block of frames and the summaries are merged by integer all-reduce; the
merged count map, histograms and hit list equal those of processing every
frame at once.  The per-rank processing is the oracle here (no GPU)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1903_06838_gb300 import dist as pdist  # noqa: E402
from paper_1903_06838_gb300 import synth  # noqa: E402
from tests._cases import sort_hits  # noqa: E402

DET = synth.Detector(n_modules=2, rows=24, cols=40, unit_rows=24, unit_cols=20,
                     occupancy=0.03, seed=9)
N_FRAMES = 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    ped, gain = synth.maps(DET)
    raw, _ = synth.frames(DET, ped, gain, 0, N_FRAMES, truth=False)
    return ped, gain, raw


def _rank(rank, ws, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ped, gain, raw = _inputs()
        a, b = pdist.shard(N_FRAMES, ws, rank)
        g = oracle.geometry(**DET.geometry())
        t = oracle.thresholds(**DET.thresholds())
        res = oracle.process(g, t, ped, gain, raw[a:b], frame_base=a)
        cmap, hp, hh = pdist.merge_summaries(res.count_map, res.hist_pix, res.hist_hit)
        hits = pdist.gather_hits(res.hits, res.hits.dtype)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), cmap=cmap, hp=hp, hh=hh,
                 hits=hits.view(np.uint8))
    finally:
        dist.destroy_process_group()


def test_shard_covers_every_frame_once():
    for n in (0, 1, 7, 64, 1025):
        for ws in (1, 2, 3, 8):
            parts = [pdist.shard(n, ws, r) for r in range(ws)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(ws - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pdist.shard(4, 2, 2)


def test_two_ranks_merge_equals_one_pass(tmp_path):
    ws = 2
    mp.get_context("spawn")
    mp.spawn(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    ped, gain, raw = _inputs()
    ref = oracle.process(oracle.geometry(**DET.geometry()), oracle.thresholds(**DET.thresholds()),
                         ped, gain, raw)
    assert ref.n_hits > 0
    for rank in range(ws):
        z = np.load(tmp_path / f"rank{rank}.npz")
        np.testing.assert_array_equal(z["cmap"], ref.count_map.astype(np.uint64))
        np.testing.assert_array_equal(z["hp"], ref.hist_pix.astype(np.uint64))
        np.testing.assert_array_equal(z["hh"], ref.hist_hit.astype(np.uint64))
        hits = z["hits"].view(ref.hits.dtype)
        assert sort_hits(hits).tobytes() == sort_hits(ref.hits).tobytes()
