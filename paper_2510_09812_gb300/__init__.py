"""GB300-native GSPM micromagnetics step (finite elements, magnetostatics, magnetostriction).

``synth`` builds seeded synthetic inputs; ``gspm`` is the thin ctypes binding of the CUDA
library ``libgspm.so`` (imported on demand so that input generation works without a GPU).
"""
