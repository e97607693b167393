// tma.cu -- host-side encoding of TMA tensor maps (driver entry point
// resolved at run time, so the library does not link libcuda directly).
#include <cudaTypedefs.h>

#include "glm_internal.cuh"

namespace glm {

static int encode_2d(CUtensorMap *out, const void *base, int dt, uint64_t inner, uint64_t outer,
                     uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer,
                     CUtensorMapSwizzle swz) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    GLM_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                  cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn)
      return set_error(GLM_ECUDA, "cuTensorMapEncodeTiled not available");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  CUtensorMapDataType t;
  switch (dt) {
  case GLM_F32: case GLM_TF32: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
  case GLM_BF16: t = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
  case GLM_F16: t = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
  case GLM_E4M3: t = CU_TENSOR_MAP_DATA_TYPE_UINT8; break;
  default: return set_error(GLM_EINVAL, "tensor map: bad element type");
  }
  const cuuint64_t dims[2] = {inner, outer};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(out, t, 2, const_cast<void *>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(GLM_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return GLM_OK;
}

int make_tmap_2d(CUtensorMap *out, const void *base, int dt, uint64_t inner, uint64_t outer,
                 uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  return encode_2d(out, base, dt, inner, outer, row_bytes, box_inner, box_outer,
                   CU_TENSOR_MAP_SWIZZLE_NONE);
}

int make_tmap_2d_sw128(CUtensorMap *out, const void *base, int dt, uint64_t inner,
                       uint64_t outer, uint64_t row_bytes, uint32_t box_inner,
                       uint32_t box_outer) {
  return encode_2d(out, base, dt, inner, outer, row_bytes, box_inner, box_outer,
                   CU_TENSOR_MAP_SWIZZLE_128B);
}

int make_tmap_4d_f32(CUtensorMap *out, const void *base, const uint64_t dims[4],
                     const uint64_t strides[3], const uint32_t box[4]) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  GLM_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                cudaEnableDefault, &q));
  if (q != cudaDriverEntryPointSuccess || !fn)
    return set_error(GLM_ECUDA, "cuTensorMapEncodeTiled not available");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
  const cuuint64_t st[3] = {strides[0], strides[1], strides[2]};
  const cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), d, st,
                      bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return set_error(GLM_ECUDA, "cuTensorMapEncodeTiled (4D) failed (" + std::to_string((int)r) +
                                    ")");
  return GLM_OK;
}

}  // namespace glm
