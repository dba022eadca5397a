"""GB300 (sm_103a) full-field FFT Green-operator solver with Meric-Cailletaud crystal
plasticity for polycrystalline RVEs (arXiv 2402.09996).

Importing the package loads nothing; `paper_2402_09996_gb300.rve` binds librve.so
(built by `paper_2402_09996_gb300.build_lib.build()`), and
`paper_2402_09996_gb300.inputs` draws seeded synthetic microstructures.
"""

__all__ = ["rve", "inputs", "build_lib"]
