// Single-field encode kernels for uint32 symbols (the segment path with the
// general encoder as its fallback), in a translation unit of their own so the
// three symbol widths compile in parallel.
#include "encode_seg.cuh"

namespace huff {

template <typename Sym>
EncOneFn encode_one_kernel_get(bool gtab, bool long_ok) {
    if (long_ok) return gtab ? encode_one_kernel<Sym, true, true> : encode_one_kernel<Sym, false, true>;
    return gtab ? encode_one_kernel<Sym, true, false> : encode_one_kernel<Sym, false, false>;
}

template EncOneFn encode_one_kernel_get<uint32_t>(bool, bool);

}  // namespace huff
