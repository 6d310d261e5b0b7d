"""The torch.autograd.Function over the forward render and its hand-written
adjoint (the derivative of Eq. 6 with respect to the particle positions).

* torch.autograd.grad of the L2 loss against a target render, through
  lt_render (LTRender), on the 64^3 lattice at 512^2: the gradient of the
  256 seeded particles against the oracle's FP64 gradient of the same loss
  (relative l2 within 1e-3), and the untouched fourth component of the
  float4 positions gets no gradient.
* The adjoint covers orthographic frames: lt_render_backward refuses frames
  binned with a perspective camera, whatever the atomic form rendered since.
"""
import numpy as np
import pytest

import oracle
from lt_inputs import ZeldovichField, config, ortho_z, sphere_cameras

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3206_gb300.render import Renderer
    return Renderer()


def test_autograd_through_lt_render_matches_oracle_gradient(R):
    from paper_1208_3206_gb300.render import lt_render
    c = config("zel64_grad512")
    N, W, H = c["N"], c["W"], c["H"]
    pos_np = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["seed"]).positions(c["lams"][0])
    tpos = ZeldovichField.generate(N, c["n_index"], c["k_cut"], c["target_seed"]).positions(c["lams"][0])
    cam = ortho_z(W, H)
    target = torch.from_numpy(oracle.render(tpos, N, cam)).cuda()
    pos = torch.from_numpy(pos_np).cuda().requires_grad_(True)
    img = lt_render(pos, N, [cam], renderer=R)
    assert img.shape == (1, H, W) and img.requires_grad
    loss = ((img[0].double() - target) ** 2).sum()
    (g,) = torch.autograd.grad(loss, pos)
    R.sync()
    assert g.shape == pos.shape and g.dtype == torch.float32
    g = g.cpu().numpy().astype(np.float64)
    assert np.all(g[:, 3] == 0.0)
    # the oracle's FP64 gradient for the same dL/dI (the one autograd passed down)
    dLdI = 2.0 * (img[0].detach().double() - target).cpu().numpy()
    g_ref = oracle.gradient(pos_np, N, cam, dLdI)
    parts = np.random.default_rng(c["grad_seed"]).choice(N ** 3, size=c["grad_particles"], replace=False)
    a, b = g[parts, :3].ravel(), g_ref[parts].ravel()
    assert np.linalg.norm(b) > 0
    assert np.linalg.norm(a - b) <= GRAD_TOL * np.linalg.norm(b)


def test_backward_checks_the_binned_frames_not_the_last_atomic_render(R):
    from paper_1208_3206_gb300._lib import LtError
    N, W = 16, 64
    pos = torch.from_numpy(ZeldovichField.generate(N, -2.0, 6.0, 41).positions(1.2)).cuda()
    persp = sphere_cameras(3, W, W)[1]
    ortho = ortho_z(W, W)
    g = torch.ones((1, W, W), dtype=torch.float32, device="cuda")
    R.build_tets(pos, N)
    # perspective frames binned, then the atomic form renders an orthographic view
    R.project_bin([persp])
    R.render_atomic([ortho])
    with pytest.raises(LtError) as e:
        R.render_backward(g)
    assert e.value.name == "LT_ERR_ARG"
    # orthographic frames binned, then the atomic form renders a perspective view
    R.project_bin([ortho])
    R.render_atomic([persp])
    out = R.render_backward(g)
    R.sync()
    assert torch.isfinite(out).all()
