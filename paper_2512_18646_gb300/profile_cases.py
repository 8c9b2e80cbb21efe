"""Small cases of the hot kernels, sized for profiler captures.

`python -m paper_2512_18646_gb300.profile_cases <case>` runs one case on
cuda:0 through the library. The cases use the CNN parameter set (N = 2^16,
Q = 60 + 12 x 45, P = 2 x 60, digits of two primes) on a narrow image slab, so
every launch has the shape of the full workload's launches per limb while the
device holds a few GB at most and each launch's data exceeds L2:

  conv1   16 image columns (16 ciphertexts of 128 pixels, 256 images):
          hoisted rotations by 1..4 (ModUp NTTs over 16 x 7 x 15 limbs,
          key inner products, ModDown) then the 8-channel 5x5 stride-2 MAC
          and rescale.
  square  the x^2 activation (tensor, relinearisation, rescale) of 64
          ciphertexts at the top level (13 limbs).
  conv2   the second convolution (16 x 3 x 3 stride 2 over 8 channels of 16
          columns, row gap 2) on 128 ciphertexts at 11 limbs.
  fc      the dense layer's plaintext multiply-accumulate, rescale and
          rotate-and-add on 16 x 4 input ciphertexts at 9 limbs, 10 outputs.

The case body (after key generation and encryption) runs inside the NVTX
range "case", so a capture can be limited to it (ncu --nvtx --nvtx-include
"case/").
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["conv1", "conv2", "square", "fc"])
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    from inputs import synthetic
    from paper_2512_18646_gb300 import api, load
    from paper_2512_18646_gb300._build import build
    build()
    load()
    pre = synthetic.CNN_N16
    g = api.Context.from_preset(pre, seed=5)
    g.keygen([1, 2, 3, 4])
    w = synthetic.cnn_weights(128, seed=302)
    import numpy as np
    import torch
    if args.case == "conv2":
        rng = np.random.default_rng(4)
        m = rng.integers(-(1 << 40), 1 << 40, size=(8 * 16, g.N), dtype=np.int64)
        x = g.encrypt_coeffs(m, 11, g.scale)
    elif args.case == "fc":
        g.keygen([4, 8, 16, 32, 64])
        rng = np.random.default_rng(3)
        m = rng.integers(-(1 << 40), 1 << 40, size=(64, g.N), dtype=np.int64)
        x = g.encrypt_coeffs(m, 9, g.scale)
        W = rng.normal(0, 0.05, (10, 16 * 30 * 4))
        pts = g.fc_prepare(W, 16, 30, 4, 4, 128, 256, 9)
    else:
        imgs = synthetic.images(256, 128, 16 if args.case == "conv1" else 64, seed=301)
        x = g.encrypt_image(imgs, 128)
    g.synchronize()
    torch.cuda.nvtx.range_push("case")
    for _ in range(args.repeat):
        if args.case == "conv1":
            y = g.conv2d(x, 1, 1, w.conv1_w, w.conv1_b, 2)
        elif args.case == "conv2":
            y = g.conv2d(x, 8, 2, w.conv2_w, w.conv2_b, 2)
        elif args.case == "fc":
            y = g.fc_apply(x, pts, None)
        else:
            y = g.mul(x, x)
        del y
    g.synchronize()
    torch.cuda.nvtx.range_pop()
    print(f"profile case {args.case} done")


if __name__ == "__main__":
    main()
