"""The learned count / subpixel network on the GPU: forward outputs and
every parameter gradient against the float64 CPU oracle (oracle/net.py), the
patch gather against the oracle's corrected frames, and a short training run
on generated hits that must beat the classical centre of mass."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import net as onet
from paper_1903_06838_gb300 import learn, pd, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _random_batch(rng, B):
    x = rng.normal(0.0, 0.3, (B, 25))
    x[:, 12] += rng.uniform(0.3, 3.0, B)
    counts = rng.integers(0, 5, B).astype(np.uint8)
    tgt = rng.uniform(-0.5, 0.5, (B, 2)).astype(np.float32)
    mask = (rng.random(B) < 0.7).astype(np.uint8)
    return x.astype(np.float32), counts, tgt, mask


def _params(seed):
    P = onet.init_params(seed)
    flat = onet.flatten(P).astype(np.float32)
    return onet.unflatten(flat.astype(np.float64)), flat


def test_forward_matches_oracle_with_bf16_operands():
    rng = np.random.default_rng(0)
    P, flat = _params(1)
    net = pd.pd_net_create(4096, seed=0)
    pd.pd_net_set_params(net, flat)
    x, *_ = _random_batch(rng, 3000)
    got = learn.predict(net, torch.from_numpy(x).cuda()).cpu().numpy()
    ref, _ = onet.forward(P, x.astype(np.float64), operand=onet.bf16)
    np.testing.assert_allclose(got, ref, rtol=2e-3, atol=2e-3)
    exact, _ = onet.forward(P, x.astype(np.float64))
    assert np.abs(got - exact).max() < 0.05  # bfloat16 operands stay close


def test_forward_full_size_sampled_against_oracle():
    """2^17 + 1000 patches through chunks of 65 536 (each CTA runs several
    conv and FC tiles, the TMEM buffers and mbarrier phases wrap, the next
    tile's patches are prefetched, and the call crosses a chunk boundary with
    a ragged tail): every 61st hit, which covers every CTA's later tiles,
    equals the float64 oracle with the same bf16 operand rounding.  The
    forward pass is per hit, so the oracle on the sample is exact."""
    rng = np.random.default_rng(5)
    P, flat = _params(4)
    net = pd.pd_net_create(65536, seed=0)
    pd.pd_net_set_params(net, flat)
    n = (1 << 17) + 1000
    x, *_ = _random_batch(rng, n)
    got = learn.predict(net, torch.from_numpy(x).cuda()).cpu().numpy()
    idx = np.arange(0, n, 61)
    idx = np.union1d(idx, np.arange(n - 64, n))  # the ragged tail in full
    ref, _ = onet.forward(P, x[idx].astype(np.float64), operand=onet.bf16)
    np.testing.assert_allclose(got[idx], ref, rtol=2e-3, atol=2e-3)
    assert np.isfinite(got).all()


# 1024 hits: one 8-hit tile per CTA of the convolution kernels; 3001: CTAs
# loop over several tiles and the last tile holds one hit
@pytest.mark.parametrize("n_hits", [1024, 3001])
def test_gradients_match_float64_oracle(n_hits):
    rng = np.random.default_rng(2)
    P, flat = _params(3)
    net = pd.pd_net_create(4096, seed=0)
    pd.pd_net_set_params(net, flat)
    x, counts, tgt, mask = _random_batch(rng, n_hits)
    dev = [torch.from_numpy(a).cuda() for a in (x, counts, tgt, mask)]
    grads = torch.zeros(pd.pd_net_num_params(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    nreg = float(mask.sum())
    pd.pd_net_gradients(net, *(d.data_ptr() for d in dev), len(x), nreg, 10.0,
                        grads.data_ptr(), loss.data_ptr())
    torch.cuda.synchronize()
    # The only approximation of the GPU path is the bfloat16 rounding of the
    # two operands of every contraction (float32 accumulation): against the
    # oracle with the same operand rounding the gradients agree to the
    # float32 accumulation level; against exact float64 the bfloat16 error
    # (2^-9 relative per operand, compounded through the backward chain)
    # bounds the difference.
    ref_loss, ref_g, _ = onet.loss_and_grad(P, x.astype(np.float64), counts, tgt, mask, 10.0)
    _, mir_g, _ = onet.loss_and_grad(P, x.astype(np.float64), counts, tgt, mask, 10.0,
                                     operand=onet.bf16)
    assert abs(loss.item() - ref_loss) < 1e-2 * abs(ref_loss)
    got = onet.unflatten(grads.cpu().numpy().astype(np.float64))
    for k in onet.ORDER:
        a, b, c = got[k].ravel(), ref_g[k].ravel(), mir_g[k].ravel()
        rel_mirror = np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-12)
        rel_exact = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel_mirror < 5e-3, (k, rel_mirror)
        assert rel_exact < 5e-2 and cos > 0.999, (k, rel_exact, cos)


def test_gather_equals_oracle_corrected_patches():
    det = synth.asic_352x384(rows=64, occupancy=0.02)
    ped, gain = synth.maps(det)
    raw, _ = synth.frames(det, ped, gain, 0, 3)
    ctx = pd.pd_create(det.geometry(), ped, gain, det.thresholds())
    hits, patches, _ = learn.hits_and_patches(ctx, det, pd.frames_to_device(raw))
    ref = oracle.process(oracle.geometry(**det.geometry()),
                         oracle.thresholds(**det.thresholds()), ped, gain, raw,
                         want_corrected=True)
    corr = ref.corrected.reshape(3, det.rows, det.cols)
    got = patches.cpu().numpy()
    ph = np.float32(det.photon_kev)
    for j, h in enumerate(hits):
        r0, c0 = divmod(int(h["pixel"]), det.cols)
        exp = np.zeros(25, np.float32)
        for k in range(25):
            r, c = r0 + k // 5 - 2, c0 + k % 5 - 2
            if 0 <= r < det.rows and 0 <= c < det.cols:
                exp[k] = corr[int(h["frame"]), r, c] / ph
        assert got[j].tobytes() == exp.tobytes()


def test_training_beats_centre_of_mass():
    """A few hundred Adam steps on hits with known truth (occupancy up to
    5 %, cloud width U(0.2, 0.5) px): on held-out single-photon hits the
    learned offsets have a smaller RMS error than the classical centre of
    mass, and the refined hits keep the classical values where the network
    is not confident."""
    det = synth.asic_352x384(occupancy=0.005, occupancy_hi=0.05, cloud_sigma=0.2,
                             cloud_sigma_hi=0.5, seed=31)
    _, ptr, (c_tr, *_), lab_tr = learn.make_set(det, 40, 0)
    hits_te, pte, (c_te, t_te, m_te), _ = learn.make_set(det, 12, 1000)
    net = pd.pd_net_create(4096, seed=7)
    losses = learn.train(net, ptr, lab_tr, steps=800, batch=2048, lr=2e-3)
    assert np.mean(losses[-20:]) < 0.6 * np.mean(losses[:5])
    out = learn.predict(net, pte).cpu().numpy()
    single = m_te == 1
    com = np.stack([hits_te["dx"], hits_te["dy"]], 1)[single]
    learned = out[single, 5:7]
    rms_com = np.sqrt(((com - t_te[single]) ** 2).mean())
    rms_net = np.sqrt(((learned - t_te[single]) ** 2).mean())
    assert rms_net < rms_com, (rms_net, rms_com)
    # refinement with the confidence fallback
    outs = torch.from_numpy(out).cuda()
    hin = torch.from_numpy(hits_te.view(np.uint8).reshape(len(hits_te), 24)).cuda()
    hout = torch.empty_like(hin)
    pd.pd_net_refine(outs.data_ptr(), hin.data_ptr(), len(hits_te), 0.9, 0.9, hout.data_ptr())
    torch.cuda.synchronize()
    ref = hout.cpu().numpy().view(pd.HIT_DTYPE).reshape(-1)
    learned_flag = (ref["flags"] & pd.PD_HIT_LEARNED) != 0
    probs = np.exp(out[:, :5] - out[:, :5].max(1, keepdims=True))
    probs /= probs.sum(1, keepdims=True)
    confident = (probs.max(1) >= 0.9) & (probs.argmax(1) >= 1)
    clear = np.abs(probs.max(1) - 0.9) > 1e-4  # float32 sums may differ at the edge
    np.testing.assert_array_equal(learned_flag[clear], confident[clear])
    keep = ~learned_flag
    assert (ref["dx"][keep] == hits_te["dx"][keep]).all()
    assert (ref["count"][learned_flag] == probs.argmax(1)[learned_flag]).all()
    # a count gate above 1 keeps every classical count, offsets still refined
    pd.pd_net_refine(outs.data_ptr(), hin.data_ptr(), len(hits_te), 0.9, 2.0, hout.data_ptr())
    torch.cuda.synchronize()
    ref2 = hout.cpu().numpy().view(pd.HIT_DTYPE).reshape(-1)
    assert (ref2["count"] == hits_te["count"]).all()
    assert (ref2["dx"] == ref["dx"]).all() and (ref2["flags"] == ref["flags"]).all()
