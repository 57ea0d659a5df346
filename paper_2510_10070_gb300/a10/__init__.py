"""Measurement of the tensor-core radix-16 option (see dft16_mma.cu)."""
