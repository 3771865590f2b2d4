"""GB300-native batched evaluator of the polar AC optimal power flow model (ExaGO, arXiv 2203.10587).

The package holds the seeded synthetic-grid generator (``synth``), the C-ABI library sources
(``csrc/``), the build step (``build``) and the thin ctypes binding (``exago``).  Importing the
package loads nothing; ``exago`` loads the compiled library on first use and raises if it is
missing.
"""
