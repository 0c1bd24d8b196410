// Chunk-aligned layout (HUFF_LAYOUT_CHUNK_ALIGNED) of the single-field
// encoder: encode_kernel with the padding of each chunk to a unit boundary in
// the tile scan.  Its instantiations live in a translation unit of their own,
// so the dense kernels keep code without the padding step and both compile in
// parallel.
#include "encode_impl.cuh"

namespace huff {

template <typename Sym>
EncKernelFn encode_kernel_aligned(bool gtab) {
    return gtab ? encode_kernel<Sym, true, false, true> : encode_kernel<Sym, false, false, true>;
}

template EncKernelFn encode_kernel_aligned<uint8_t>(bool);
template EncKernelFn encode_kernel_aligned<uint16_t>(bool);
template EncKernelFn encode_kernel_aligned<uint32_t>(bool);

}  // namespace huff
