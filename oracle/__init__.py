"""FP64 CPU oracle for the DASS per-timestep hot path.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of what the paper's method computes, used to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it; the product path (the C-ABI library and its Python binding) never
does, and the oracle never imports the product path. The two share no code:
the only common module is the seeded input generator, which holds none of the
method's arithmetic.

Everything here is PyTorch CPU float64 (or NumPy), each function citing the
passage of arXiv 2411.14847 ("Dynamics-Aware Gaussian Splatting Streaming")
that defines it. Gradients are obtained by reverse-mode automatic
differentiation of the forward definition (torch.autograd, a library primitive),
storing every alpha -- deliberately a different algorithm from the CUDA
backward, which recomputes alpha from the saved final transmittance.

Modules:
  gaussians  -- activations, quaternions, covariance, EWA projection, real SH (App. A.1, Sec. 3.3)
  composite  -- untiled per-pixel front-to-back alpha blending (App. A.1 Eq. for C)
  loss       -- L1 + D-SSIM fidelity loss (Eq. 2 / Eq. 3)
  stages     -- selective inheritance (Eq. 1), dynamics-aware shift (Sec. 3.3),
                masked Adam, error map + Alg. 1 projection + Eq. 4 selection + spawn (Sec. 3.4)
  binning    -- brute-force (tile, depth, index) ordering in FP32 for the tile-list check
  grad       -- end-to-end loss gradients by autograd through all of the above, the learned
                inheritance mask's straight-through gradient (Eq. 1-2)
  field      -- hash-encoding deformation fields H_dyn / H_st (Sec. 3.3, App. B.2)
  dynamics   -- identity-feature rendering and the per-Gaussian dynamics query (Sec. 3.3, App. A.2)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, library routines, brute force, invariants or finite differences,
except where its docstring says "parity unpinned".
"""
