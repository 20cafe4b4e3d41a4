"""FP64 CPU oracle of the design-objective engine.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA path is checked against.  Only the tests, the smoke check and the CPU
baseline of the benchmark may import it; the CUDA library and its Python
binding never do, and the oracle imports nothing from them.

Modules:
  mc      -- FP64 Monte Carlo with its own Philox4x32-10 (Sec. 2.2, Eq. 5-7)
  quad    -- deterministic orthant probabilities, FWER calibration (Eq. 2, 4)
  smooth  -- local-polynomial smoother and argmax (Sec. 2.3)
  design  -- design model restated independently; exact-objective gradients
"""
