"""lt_frame_mass_static, the allocation-free entry point, against the frame
mass lt_render_tiles reduces for the same images: two calls in a row, each
within 1e-12 (relative) of it and bit-identical to each other (the order of
the sums is fixed). Also its argument and capacity errors."""
import numpy as np
import pytest

from lt_inputs import ZeldovichField, camera_dict, ortho_z

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_frame_mass_static_matches_render_tiles_mass():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1208_3206_gb300._lib import LtError
    from paper_1208_3206_gb300.render import Renderer, lt_frame_mass_static

    N, W, H = 32, 256, 256
    f = ZeldovichField.generate(N, -2.0, 16.0, 1001)
    pos = np.concatenate([f.positions(1.5), f.positions(3.0)])
    # three windows of the same size (same pixel area): two periodic box
    # windows and one shifted, non-periodic one
    cams = [ortho_z(W, H), ortho_z(W, H),
            camera_dict("ortho", W, H, lo=(0.25, 0.1), hi=(1.25, 1.1), wrap=False)]
    R = Renderer()
    R.build_tets(torch.from_numpy(pos).cuda(), N)
    R.project_bin(cams, [0, 1, 1])
    img, mass = R.render_tiles(with_mass=True)
    R.sync()
    ref = mass.cpu().numpy()
    area = 1.0 / (W * H)
    first = lt_frame_mass_static(img, area).cpu().numpy()
    second = lt_frame_mass_static(img, area).cpu().numpy()
    assert np.array_equal(first, second)
    np.testing.assert_allclose(first, ref, rtol=1e-12, atol=0)
    with pytest.raises(LtError) as e:
        lt_frame_mass_static(torch.zeros((129, 2, 2), dtype=torch.float32, device="cuda"), 1.0)
    assert e.value.name == "LT_ERR_CAPACITY"
    with pytest.raises(LtError) as e:
        lt_frame_mass_static(img, 0.0)
    assert e.value.name == "LT_ERR_ARG"
