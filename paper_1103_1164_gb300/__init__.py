"""GB300-native DC-FSPB dose engine (Gu et al., arXiv 1103.1164).

The compute path is the C-ABI library ``libdc_fspb.so`` built from ``csrc/``;
``paper_1103_1164_gb300.dc_fspb`` is its Python binding.  Importing the package
itself loads nothing, so that ``synth`` (the seeded input generators) can be
used on machines without the library.
"""
