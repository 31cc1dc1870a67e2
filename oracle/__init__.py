"""CPU oracle for hybrid-dealiased convolutions (Murasko & Bowman, arXiv 2303.17510).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
link anything in this package; only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the
CUDA library: every function here is written from the paper's equations in
plain FP64 numpy (or plain C in ``direct_conv.c``) and is pinned by tests
against brute force, closed forms, invariants and the paper's worked
examples.

Modules
  direct   -- the definition: truncated linear convolution (complex, centered,
              Hermitian; 1D and separable N-D; sampled output points), for every
              mult as signed sums of binary products (the Basdevant forms of
              Section 9 have B > 1 outputs).  Exact on integer-valued inputs.
              Section 2 (problem statement), Sections 3-5.
  params   -- parameter derivation p, q, n of Alg. convolve / convolveX and the
              inner-loop redefinition (Eq. pqdef1, Section 6.1, Section 6.2);
              dealiasing bounds; work-memory formulas (Section 4/5, memory).
  residue  -- per-residue forward transforms by their definition: the length-qm
              DFT of the zero-padded (or centered) input at k = q*l + r
              (Eq. forStan, Eq. centDFT, Eq. wHerDef, Section 6.1-6.2).
  steps    -- the paper's residue-at-a-time algorithm (Alg. convolve/convolveX
              with forward1/2/Inner, centered and Hermitian variants) in the
              paper's order, with an FFT library call as the size-m FFT step;
              optionally over a residue range only (the partial sum one share
              of a residue-split convolution computes, Section 2.2).
  explicit -- explicit zero-padded FFT convolution (the paper's comparison
              method, Section 7) with numpy's FFT as the FFT step; optionally
              with the product spectrum restricted to the frequencies of a
              residue range on axis 0 (pins the residue partial sums).
  cdirect  -- ctypes wrapper of direct_conv.c, the same definition in plain C
              (multithreaded over instances) for large samples and CPU timing.
  mlp      -- FP64 reference of the parameter-selector MLP (forward, backward,
              SGD step) used to check the GPU training kernels' gradients.
"""
