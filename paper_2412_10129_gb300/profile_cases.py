"""Small workloads for profiler captures of single kernels (inputs above the
129 MB L2, a few GB on the device, one launch each).

    python -m paper_2412_10129_gb300.profile_cases solvers

runs, on the half-resolution scan (256^3 at 1 mm, 360 views, 384 x 512
detector): one Siddon transpose (k_bp_siddon_scatter), one Hamming-window
FDK row filter (k_fdk_rows<1>), and one TV descent step on a 512^3 volume
(k_tv_march: norm pass, step pass).
"""
import sys


def solvers() -> None:
    import torch

    from . import build, inputs, tg
    build.build()
    tg.load()
    g = inputs.circular_geometry((256, 256, 256), (1.0,) * 3, (512, 384), (0.8, 0.8), 360, 1000.0, 1536.0)
    b = torch.rand(g.proj_shape, device="cuda")
    v = torch.empty(g.vol_shape, device="cuda")
    tg.backproject(g, b, "siddon", out=v)
    x = torch.rand((512, 512, 512), device="cuda")
    tg.tv_descent(x, 1, 1e-3)
    f = torch.empty_like(b)
    tg.fdk_filter(g, b, "hamming", out=f)
    torch.cuda.synchronize()
    print("ok")


CASES = {"solvers": solvers}

if __name__ == "__main__":
    CASES[sys.argv[1] if len(sys.argv) > 1 else "solvers"]()
