"""The continuous-batching server on the GPU: every served mask is byte-identical
to the mask of a lone fx_extract call on the same image, with requests of both
dtypes and uneven sizes mixed in batches, a budget that makes requests wait,
and batches launched while earlier ones are still running."""
import numpy as np
import pytest

from gen import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def test_served_masks_equal_alone(cuda_lib):
    from paper_1304_3992_gb300.serve import Server, TorchBackend, run_stream
    fx = cuda_lib
    p = fx.make_params(fx.FX_U16, 12)
    rng = np.random.default_rng(4)
    m8 = scenes.scene(900, 700, seed=41, n_rects=100, noise_sigma=4, impulse_frac=0.01, bits=8)
    m16 = scenes.scene(900, 700, seed=42, n_rects=100, noise_sigma=24, impulse_frac=0.005, bits=12)
    imgs = []
    for i in range(12):
        h, w = int(rng.integers(30, 600)), int(rng.integers(30, 800))
        src = m8 if i % 2 == 0 else m16
        imgs.append(_pinned(src[:h, :w]))
    be = TorchBackend(p, slots=2, max_images=16)
    budget = sum(sorted(im.nbytes + im.size for im in imgs)[-3:])  # a few requests at a time
    s = Server(be, budget_bytes=budget, max_batch=8)
    got = {}
    reqs = run_stream(s, imgs, rate_hz=3000, duration_s=0.02, seed=5,
                      on_done=lambda r: got.__setitem__(r.rid, r.dev["out"].cpu().numpy()))
    assert len(reqs) >= 10 and all(r.state == "done" for r in reqs)
    for r in reqs:
        alone = fx.extract(torch.from_numpy(r.image).cuda(), p).cpu().numpy()
        assert np.array_equal(got[r.rid], alone), f"request {r.rid} differs from the lone call"
    assert s.used == 0
    be.close()


def test_batches_overlap_on_the_device(cuda_lib):
    """A batch of small requests is launched while the big request's batch is
    still executing (its event pending at launch time: two median levels of
    radius 2 run on the general kernel, some milliseconds on 8192^2), and
    every mask equals the lone call's."""
    from paper_1304_3992_gb300.serve import Server, TorchBackend
    fx = cuda_lib
    p = fx.make_params(fx.FX_U16, 12, hmf=(5, 5))
    big = _pinned(scenes.scene(8192, 8192, seed=43, n_rects=1600, noise_sigma=24, impulse_frac=0.005, bits=12))
    small = [_pinned(big[:300 + 10 * i, :200 + 7 * i]) for i in range(4)]
    be = TorchBackend(p, slots=2, max_images=8)
    s = Server(be, budget_bytes=10**10, max_batch=8)
    r0 = s.submit(0, big)
    while r0.state != "running":
        s.step()
    rs = [s.submit(1 + i, im) for i, im in enumerate(small)]
    while any(r.state in ("pending", "copying", "ready") for r in rs):
        s.step()
    s.drain(release=False)
    assert s.overlapped_launches >= 1
    for r in [r0] + rs:
        alone = fx.extract(torch.from_numpy(r.image).cuda(), p)
        assert torch.equal(r.dev["out"], alone)
        s.release(r)
    assert s.used == 0
    be.close()
