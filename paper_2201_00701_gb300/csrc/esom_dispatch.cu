// Maps (D, list capacity) to the kernel instantiation compiled for it.
#include "esom_kernels.h"
#include "esom_variants.h"

namespace esom {

#define ESOM_DECLARE_D(DV) const KernelOps *kernel_ops_d##DV(int kc);
ESOM_DECLARE_D(4) ESOM_DECLARE_D(8) ESOM_DECLARE_D(12) ESOM_DECLARE_D(16)
ESOM_DECLARE_D(20) ESOM_DECLARE_D(24) ESOM_DECLARE_D(28) ESOM_DECLARE_D(32)
ESOM_DECLARE_D(36) ESOM_DECLARE_D(40) ESOM_DECLARE_D(44) ESOM_DECLARE_D(48)
ESOM_DECLARE_D(52) ESOM_DECLARE_D(56) ESOM_DECLARE_D(60) ESOM_DECLARE_D(64)

const KernelOps *kernel_ops(int D, int kc) {
    switch (D) {
        case 4: return kernel_ops_d4(kc);
        case 8: return kernel_ops_d8(kc);
        case 12: return kernel_ops_d12(kc);
        case 16: return kernel_ops_d16(kc);
        case 20: return kernel_ops_d20(kc);
        case 24: return kernel_ops_d24(kc);
        case 28: return kernel_ops_d28(kc);
        case 32: return kernel_ops_d32(kc);
        case 36: return kernel_ops_d36(kc);
        case 40: return kernel_ops_d40(kc);
        case 44: return kernel_ops_d44(kc);
        case 48: return kernel_ops_d48(kc);
        case 52: return kernel_ops_d52(kc);
        case 56: return kernel_ops_d56(kc);
        case 60: return kernel_ops_d60(kc);
        case 64: return kernel_ops_d64(kc);
        default: return nullptr;
    }
}

#define ESOM_DECLARE_TC_D(DV) const TcOps *tc_ops_d##DV(int kc, int prec);
ESOM_DECLARE_TC_D(4) ESOM_DECLARE_TC_D(8) ESOM_DECLARE_TC_D(12) ESOM_DECLARE_TC_D(16)
ESOM_DECLARE_TC_D(20) ESOM_DECLARE_TC_D(24) ESOM_DECLARE_TC_D(28) ESOM_DECLARE_TC_D(32)
ESOM_DECLARE_TC_D(36) ESOM_DECLARE_TC_D(40) ESOM_DECLARE_TC_D(44) ESOM_DECLARE_TC_D(48)
ESOM_DECLARE_TC_D(52) ESOM_DECLARE_TC_D(56) ESOM_DECLARE_TC_D(60) ESOM_DECLARE_TC_D(64)

const TcOps *tc_ops(int D, int kc, int prec) {
    switch (D) {
        case 4: return tc_ops_d4(kc, prec);
        case 8: return tc_ops_d8(kc, prec);
        case 12: return tc_ops_d12(kc, prec);
        case 16: return tc_ops_d16(kc, prec);
        case 20: return tc_ops_d20(kc, prec);
        case 24: return tc_ops_d24(kc, prec);
        case 28: return tc_ops_d28(kc, prec);
        case 32: return tc_ops_d32(kc, prec);
        case 36: return tc_ops_d36(kc, prec);
        case 40: return tc_ops_d40(kc, prec);
        case 44: return tc_ops_d44(kc, prec);
        case 48: return tc_ops_d48(kc, prec);
        case 52: return tc_ops_d52(kc, prec);
        case 56: return tc_ops_d56(kc, prec);
        case 60: return tc_ops_d60(kc, prec);
        case 64: return tc_ops_d64(kc, prec);
        default: return nullptr;
    }
}

#define ESOM_DECLARE_TCD_D(DV) const TcOps *tc_dump_ops_d##DV(int prec);
ESOM_DECLARE_TCD_D(4) ESOM_DECLARE_TCD_D(8) ESOM_DECLARE_TCD_D(12) ESOM_DECLARE_TCD_D(16)
ESOM_DECLARE_TCD_D(20) ESOM_DECLARE_TCD_D(24) ESOM_DECLARE_TCD_D(28) ESOM_DECLARE_TCD_D(32)
ESOM_DECLARE_TCD_D(36) ESOM_DECLARE_TCD_D(40) ESOM_DECLARE_TCD_D(44) ESOM_DECLARE_TCD_D(48)
ESOM_DECLARE_TCD_D(52) ESOM_DECLARE_TCD_D(56) ESOM_DECLARE_TCD_D(60) ESOM_DECLARE_TCD_D(64)

const TcOps *tc_dump_ops(int D, int prec) {
    switch (D) {
        case 4: return tc_dump_ops_d4(prec);
        case 8: return tc_dump_ops_d8(prec);
        case 12: return tc_dump_ops_d12(prec);
        case 16: return tc_dump_ops_d16(prec);
        case 20: return tc_dump_ops_d20(prec);
        case 24: return tc_dump_ops_d24(prec);
        case 28: return tc_dump_ops_d28(prec);
        case 32: return tc_dump_ops_d32(prec);
        case 36: return tc_dump_ops_d36(prec);
        case 40: return tc_dump_ops_d40(prec);
        case 44: return tc_dump_ops_d44(prec);
        case 48: return tc_dump_ops_d48(prec);
        case 52: return tc_dump_ops_d52(prec);
        case 56: return tc_dump_ops_d56(prec);
        case 60: return tc_dump_ops_d60(prec);
        case 64: return tc_dump_ops_d64(prec);
        default: return nullptr;
    }
}

#define ESOM_DECLARE_VAR_D(DV) const VariantOps *variant_ops_d##DV();
ESOM_DECLARE_VAR_D(4) ESOM_DECLARE_VAR_D(8) ESOM_DECLARE_VAR_D(12) ESOM_DECLARE_VAR_D(16)
ESOM_DECLARE_VAR_D(20) ESOM_DECLARE_VAR_D(24) ESOM_DECLARE_VAR_D(28) ESOM_DECLARE_VAR_D(32)
ESOM_DECLARE_VAR_D(36) ESOM_DECLARE_VAR_D(40) ESOM_DECLARE_VAR_D(44) ESOM_DECLARE_VAR_D(48)
ESOM_DECLARE_VAR_D(52) ESOM_DECLARE_VAR_D(56) ESOM_DECLARE_VAR_D(60) ESOM_DECLARE_VAR_D(64)

const VariantOps *variant_ops(int D) {
    switch (D) {
        case 4: return variant_ops_d4();
        case 8: return variant_ops_d8();
        case 12: return variant_ops_d12();
        case 16: return variant_ops_d16();
        case 20: return variant_ops_d20();
        case 24: return variant_ops_d24();
        case 28: return variant_ops_d28();
        case 32: return variant_ops_d32();
        case 36: return variant_ops_d36();
        case 40: return variant_ops_d40();
        case 44: return variant_ops_d44();
        case 48: return variant_ops_d48();
        case 52: return variant_ops_d52();
        case 56: return variant_ops_d56();
        case 60: return variant_ops_d60();
        case 64: return variant_ops_d64();
        default: return nullptr;
    }
}

}  // namespace esom
