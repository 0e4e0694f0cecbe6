"""GB300-native MOMMS: multilevel-blocked FP64 dense matrix multiplication.

C := alpha * op(A) * op(B) + beta * C on column-major matrices with leading
dimensions, on one GB300 (sm_103a), through the C-ABI library ``libmomms``:

* native FP64 on the DMMA tensor instructions (C micro-tile resident in
  registers, the paper's Resident C at L0, Sec. 3.4);
* FP64 emulated by signed integer digit slices on the fp16 tcgen05 tensor
  cores with exact FP32 accumulation in tensor memory, drained into exact
  integers and recombined in FP64;
* backward (dA = dC B^T, dB = A^T dC), a batched persistent launch, and a
  plan cache that picks the family member, tile and slice count.

The binding (``momms``) loads the compiled library lazily; importing this
package does not touch the GPU.  ``synthetic`` holds the seeded input
generators.
"""

__all__ = ["momms", "synthetic"]
