"""tsplat: GB300-native latent-feature Gaussian splatting (Tele-Aloha, Sec. 4.2).

    from paper_2405_14866_gb300 import api, gen
    g = api.Gaussians.build(views, C=32, feat_dtype=api.BF16)   # A1
    ctx = api.Context()
    F, A = ctx.render(g, target_camera)                          # A2..A7

The computation runs in libtsplat.so (CUDA, sm_103a), built in-tree by
paper_2405_14866_gb300.build; this package only marshals arguments.
"""
