"""GB300-native pixel-aligned implicit occupancy field with hierarchical
surface localization and mesh-free rendering (Li et al., "Monocular Real-Time
Volumetric Performance Capture", Sec. 3.1-3.2).

Importing the package loads nothing; the CUDA library is opened by
``paper_2007_13988_gb300.pifu`` on first use.
"""
