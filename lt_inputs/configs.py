"""The five synthetic workloads, by name. Each stands in for a simulation
snapshot of the paper's kind (a deformed particle lattice with shell
crossing) at the stated lattice size, view and image size."""
from __future__ import annotations

CONFIGS = {
    # 32^3 particles, 196,608 tets, orthographic along z, 256^2 px
    "zel32_ortho256": dict(N=32, n_index=-2.0, k_cut=16.0, lams=[1.5], seed=1001,
                           view="ortho_z", W=256, H=256),
    # 128^3 particles, 12.6M tets, orthographic along z, 1024^2 px
    "zel128_ortho1024": dict(N=128, n_index=-2.5, k_cut=48.0, lams=[3.0], seed=1002,
                             view="ortho_z", W=1024, H=1024),
    # 256^3 particles, 100.7M tets, 8 snapshots x 16 perspective cameras, 2048^2 px
    "zel256_persp2048x128": dict(N=256, n_index=-2.5, k_cut=96.0,
                                 lams=[0.5 + i * (6.0 - 0.5) / 7 for i in range(8)], seed=1003,
                                 view="sphere16", W=2048, H=2048, radius=2.0, fov_y_deg=60.0),
    # 512^3 particles, 805M tets, float16 offsets, orthographic along z, 4096^2 px
    "zel512_fp16_ortho4096": dict(N=512, n_index=-2.5, k_cut=192.0, lams=[8.0], seed=1004,
                                  view="ortho_z", W=4096, H=4096, fp16=True, crops=64,
                                  crop_size=256, crop_seed=4004),
    # 64^3 particles, 1.57M tets, L2 loss against a differently seeded target at 512^2 px
    "zel64_grad512": dict(N=64, n_index=-2.5, k_cut=24.0, lams=[2.0], seed=1005, target_seed=2005,
                          view="ortho_z", W=512, H=512, grad_particles=256, grad_seed=5005),
}


def config(name: str) -> dict:
    return dict(CONFIGS[name])
