// Drives the host-side paths of the C ABI that run without a GPU: argument validation of the
// product, level-3 and step entry points, null handles, handle creation failing cleanly when no
// device exists, the moduli planning call over its whole range, the tile-order queries and the
// status strings.  Built with AddressSanitizer / UndefinedBehaviorSanitizer from the library's
// sources by tests/test_sanitize_cpu.py; any finding ends the process with a report.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>

#include "momms.h"

static int fails = 0;
#define CHECK(cond)                                                            \
    do {                                                                       \
        if (!(cond)) {                                                         \
            std::fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            ++fails;                                                           \
        }                                                                      \
    } while (0)

static double* fake(int64_t slot) {  // a non-null address never dereferenced: validation comes first
    return reinterpret_cast<double*>(static_cast<uintptr_t>(1ull << 40) + static_cast<uintptr_t>(slot) * (1ull << 30));
}

int main() {
    // BLAS-style argument indices of the product
    CHECK(momms_gemm(-1, 2, 3, 1.0, fake(1), 1, fake(2), 3, 0.0, fake(3), 1, nullptr) == -1);
    CHECK(momms_gemm(2, -2, 3, 1.0, fake(1), 2, fake(2), 3, 0.0, fake(3), 2, nullptr) == -2);
    CHECK(momms_gemm(2, 2, -3, 1.0, fake(1), 2, fake(2), 3, 0.0, fake(3), 2, nullptr) == -3);
    CHECK(momms_gemm(4, 2, 3, 1.0, fake(1), 3, fake(2), 3, 0.0, fake(3), 4, nullptr) == -6);
    CHECK(momms_gemm(4, 2, 3, 1.0, fake(1), 4, fake(2), 2, 0.0, fake(3), 4, nullptr) == -8);
    CHECK(momms_gemm(4, 2, 3, 1.0, fake(1), 4, fake(2), 3, 0.0, fake(3), 3, nullptr) == -11);
    CHECK(momms_gemm(4, 2, 3, 1.0, nullptr, 4, fake(2), 3, 0.0, fake(3), 4, nullptr) == -5);
    CHECK(momms_gemm(8, 8, 8, 1.0, fake(1), 8, fake(2), 8, 0.0, reinterpret_cast<double*>(
                         reinterpret_cast<char*>(fake(1)) + 64), 8, nullptr) == -10);   // C overlaps A
    // null handles
    CHECK(momms_set_mode(nullptr, 1) == MOMMS_ERR_HANDLE);
    CHECK(momms_gemm_ex(nullptr, 0, 0, 1, 1, 1, 1.0, fake(1), 1, fake(2), 1, 0.0, fake(3), 1, nullptr) ==
          MOMMS_ERR_HANDLE);
    CHECK(momms_syrk(nullptr, 0, 0, 4, 4, 1.0, fake(1), 4, 0.0, fake(2), 4, nullptr) == MOMMS_ERR_HANDLE);
    CHECK(momms_trmm(nullptr, 0, 0, 0, 0, 4, 4, 1.0, fake(1), 4, fake(2), 4, nullptr) == MOMMS_ERR_HANDLE);
    CHECK(momms_trsm(nullptr, 0, 0, 0, 0, 4, 4, 1.0, fake(1), 4, fake(2), 4, nullptr) == MOMMS_ERR_HANDLE);
    momms_report_t rep;
    CHECK(momms_get_last_report(nullptr, &rep) == MOMMS_ERR_HANDLE);
    CHECK(momms_destroy(nullptr) != MOMMS_OK);
    // handle creation: succeeds with a device, fails cleanly (nothing leaked) without one
    momms_handle_t h = nullptr;
    const int rc = momms_create(&h);
    CHECK(rc == MOMMS_OK || (rc == MOMMS_ERR_ALLOC && h == nullptr));
    if (rc == MOMMS_OK) CHECK(momms_destroy(h) == MOMMS_OK);
    CHECK(momms_create(nullptr) == -1);
    // the moduli over the whole (bits, k) range
    uint32_t moduli[16];
    int count = 0;
    for (int bits = 0; bits <= 60; ++bits)
        for (int64_t k : {int64_t(0), int64_t(1), int64_t(63), int64_t(64), int64_t(4096), int64_t(133120),
                          int64_t(133121), int64_t(1) << 40}) {
            std::memset(moduli, 0, sizeof(moduli));
            const int r = momms_crt_moduli(bits, k, &count, moduli);
            CHECK(r == MOMMS_OK || r < 0 || r == MOMMS_ERR_UNSUPPORTED);
            if (r == MOMMS_OK) CHECK(count >= 1 && count <= 16 && moduli[0] == 255u);
        }
    // the tile orders
    int tm = 0, tn = 0;
    int64_t cnt = 0;
    for (int uplo = 0; uplo < 2; ++uplo)
        for (int width : {96, 192})
            for (int64_t n : {int64_t(0), int64_t(1), int64_t(127), int64_t(128), int64_t(1000), int64_t(65536)}) {
                CHECK(momms_tri_tile(uplo, width, n, 0, &tm, &tn, &cnt) >= 0);
                if (cnt > 0) {
                    CHECK(momms_tri_tile(uplo, width, n, cnt - 1, &tm, &tn, nullptr) == 1);
                    CHECK(momms_tri_tile(uplo, width, n, cnt, &tm, &tn, nullptr) == 0);
                }
            }
    for (int member = 0; member <= 4; ++member)
        for (int64_t ctas : {int64_t(1), int64_t(38), int64_t(152)})
            for (int64_t i = 0; i < 40; ++i)
                CHECK(momms_member_tile(member, 0, ctas - 1, ctas, i, 64, 43, &tm, &tn) >= 0);
    CHECK(momms_member_tile(9, 0, 0, 1, 0, 1, 1, &tm, &tn) < 0);
    // status strings for every code
    for (int s = -20; s <= 1010; ++s) CHECK(momms_status_string(s) != nullptr);
    if (fails) {
        std::fprintf(stderr, "%d checks failed\n", fails);
        return 1;
    }
    std::printf("abi driver: all calls clean\n");
    return 0;
}
