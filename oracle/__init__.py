"""CPU oracle for epsilon-relative Gaussian summation.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import anything from this package.  It shares
no code with the CUDA path (paper_1206_6857_gb300) and never imports it.

Modules:
  exhaustive  -- FP64 compensated exhaustive sum (the definition, Section 1)
  series      -- FP64 multi-index Hermite/Taylor algebra (Sections 2-4)
  lscv        -- least-squares cross-validation score from exact sums (Section 7)
  dualtree    -- CPU restatement of the kd-tree, the frontier decisions and the
                 FP64 estimate (Sections 5-6, Figs. 6-8)
  mlp         -- pair-selector network: FP64 forward / backward, Adam, and the
                 FP32 inference the traversal uses (not in the paper)
"""
