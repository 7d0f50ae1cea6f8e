"""Device-side inference of the trained surrogate ensemble, for profiling.

    python -m paper_1610_03484_gb300.profile_surrogate [n_points] [calls]

loads the stored weights of the 24x24x8, p = 2 class, forms the features of
n_points seeded Gauss points (default 1048576) and runs rve_surrogate_predict_dev
`calls` times (default 3) on device buffers; prints the device time of each call
(CUDA events on the context's stream) and the GEMM rate it implies.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import rve_inputs as ri  # noqa: E402
import paper_1610_03484_gb300 as rve  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_24x24x8_p2.npz")


def main(argv):
    n = int(argv[1]) if len(argv) > 1 else 1 << 20
    calls = int(argv[2]) if len(argv) > 2 else 3
    stream = torch.cuda.current_stream()
    ctx = rve.Context(precision=rve.PREC_MIXED, stream=stream.cuda_stream)
    z = np.load(WEIGHTS)
    s = rve.Surrogate(ctx, members=int(z["members"]), seed=0)
    s.set_params(z["params"])
    xyz, tets, ph, tg = ri.weave_rve(24, 24, 8)
    m = ctx.mesh_load(xyz, tets, 2, ph, tg)
    m.set_materials(ri.NOMINAL_MATRIX, ri.NOMINAL_YARN)
    T, c, t, _, _ = ri.gauss_point_states(n, 5)
    feat = torch.tensor(ctx.features(m, T, c, t), dtype=torch.float64, device="cuda")
    out = [torch.empty((n, k), dtype=torch.float64, device="cuda") for k in (36, 9, 9)]
    sp = torch.empty(n, dtype=torch.float64, device="cuda")
    flops = 2.0 * n * int(z["members"]) * (64 * 256 + 3 * 256 * 256 + 256 * 64)
    for call in range(calls):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.predict_dev(n, feat.data_ptr(), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), sp.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print(f"call {call}: {ms:.3f} ms, {flops / ms / 1e9:.1f} TFLOP/s over the ensemble's GEMMs")
    s.free()
    m.free()
    ctx.close()


if __name__ == "__main__":
    main(sys.argv)
